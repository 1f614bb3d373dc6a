"""Mixed-precision path (FP32 stencils and sources on centre-referenced
hi/lo differences, FP64 RK4 accumulation and end-of-step constraints)
against the FP64 oracle through the C ABI.  The tolerances are FP32-sized and
stated per test: the RHS relative to each field's RHS scale, the step relative
to the change the step makes."""
import numpy as np
import pytest

import initial_data as idd
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild
from tests.gpu_common import grid_for, rel_err

skbuild.build()


def _change_err(v, vo, u0, g=3):
    """Per-field max |v - vo| over the max change |vo - u0| of the step."""
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    d = np.abs(v[a] - vo[a]).max(axis=(1, 2, 3))
    s = np.abs(vo[a] - u0[a]).max(axis=(1, 2, 3))
    return np.where(s > 0, d / np.where(s > 0, s, 1.0), d)


def test_mixed_rhs_puncture():
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    g = grid_for([p], precision=1)
    g.upload_fields(0, u)
    r = g.rhs(0)
    ro = oracle.rhs(p, u, oracle.Params())
    e = rel_err(r, ro)
    print("mixed RHS rel err per field:", " ".join("%.1e" % x for x in e))
    assert e.max() <= 1e-4, dict(zip(idd.FIELD_NAMES, e))


def test_mixed_rhs_gauge_wave():
    p = idd.Patch(n=(32, 4, 4), dx=1 / 32, origin=(-0.5, -2 / 32, -2 / 32))
    g = grid_for([p], lapse=1, shift=1, bc=1, precision=1, courant=0.25)
    u = oracle.fill_periodic(p, idd.gauge_wave(p, 0.01))
    g.upload_fields(0, u)
    r = g.rhs(0)
    ro = oracle.rhs(p, u, oracle.Params(lapse=1, shift=1))
    e = rel_err(r, ro, floor=1e-3)
    assert e.max() <= 1e-4, dict(zip(idd.FIELD_NAMES, e))


def test_mixed_rk4_step_puncture():
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    g = grid_for([p], precision=1)
    g.upload_fields(0, u)
    dt = 0.5 * p.dx
    g.rk4_step(0, dt)
    v = g.download_fields(0)
    vo = oracle.rk4_step(p, u, dt, oracle.Params())
    e = _change_err(v, vo, u)
    print("mixed step err / step change per field:", " ".join("%.1e" % x for x in e))
    assert e.max() <= 1e-4, dict(zip(idd.FIELD_NAMES, e))


def test_mixed_pi_symmetry_bitwise():
    p = idd.single_puncture_patch(32, 8.0)
    g = grid_for([p], precision=1)
    g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)], noise_amp=1e-6, seed=idd.PUNCTURE_SEED, symmetrise_pi=True)
    for _ in range(3):
        g.rk4_step(0)
        assert g.pi_symmetry(0) == 0.0


def test_mixed_level_step_small_hierarchy():
    h = idd.small_binary()
    states = idd.hierarchy_data(h, noise=1e-10)
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=1))
    for i, u in enumerate(states):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    g.level_step(0)
    bo.level_step(0)
    for i in range(len(h.patches)):
        e = _change_err(g.download_fields(i), bo.current(i), states[i])
        assert e.max() <= 1e-4, (i, dict(zip(idd.FIELD_NAMES, e)))
