"""Equatorial reflection symmetry on the GPU (Sec. 2.2.2: only z >= 0 is
evolved, the z < 0 ghosts mirror z > 0): parity with the oracle's half-domain
evolution (FP64 1e-12 per RK4 step, 1e-10 per coarse step of the hierarchy;
mixed precision 1e-4 of the step's change), and the half domain equal to the
upper half of the full-domain GPU evolution of symmetric data."""
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
from tests.gpu_common import rel_err

skbuild.build()


def _symmetric_puncture(n=32):
    p = idd.centred_patch(n, 0.5)
    u = idd.add_noise(p, idd.punctures(p, [1.0], [(0.0, 0.0, 0.0)]), 1e-6, idd.PUNCTURE_SEED)
    return p, idd.symmetrise_z(p, u)


def _change_err(v, vo, u0, g=3):
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    d = np.abs(v[a] - vo[a]).max(axis=(1, 2, 3))
    s = np.abs(vo[a] - u0[a]).max(axis=(1, 2, 3))
    return np.where(s > 0, d / np.where(s > 0, s, 1.0), d)


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_half_domain_vs_oracle(precision):
    p, u = _symmetric_puncture()
    ph = idd.upper_half(p)
    uh = idd.upper_half_array(p, u)
    g = sk.Grid(1, ph.dx, [ph], sk.Params(zsym=1, precision=precision), stream=torch.cuda.Stream())
    g.upload_fields(0, uh)
    dt = 0.25 * p.dx
    uo = uh
    for _ in range(2):
        g.rk4_step(0, dt)
        uo = oracle.rk4_step(ph, uo, dt, oracle.Params(), bc=oracle.BC_SOMMERFELD | oracle.BC_ZREFLECT)
    v = g.download_fields(0)
    if precision == 0:
        assert rel_err(v, uo, active_only=True).max() <= 1e-12
    else:
        assert _change_err(v, uo, uh).max() <= 1e-4


def test_uniform_half_domain_equals_full_domain():
    p, u = _symmetric_puncture()
    ph = idd.upper_half(p)
    full = sk.Grid(1, p.dx, [p], sk.Params(), stream=torch.cuda.Stream())
    half = sk.Grid(1, ph.dx, [ph], sk.Params(zsym=1), stream=torch.cuda.Stream())
    full.upload_fields(0, u)
    half.upload_fields(0, idd.upper_half_array(p, u))
    for _ in range(3):
        full.rk4_step(0)
        half.rk4_step(0)
    a = idd.upper_half_array(p, full.download_fields(0))
    b = half.download_fields(0)
    assert rel_err(b, a, active_only=True).max() <= 1e-12


def _hierarchy():
    h = idd.small_binary(n_fixed=24, n_moving=16, n_levels=3, n_fixed_levels=2, dx0=1.0, sep=2.0)
    return h, idd.hierarchy_data(h, noise=0.0), idd.upper_half_hierarchy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_hierarchy_half_domain_vs_oracle(precision):
    h, states, hh = _hierarchy()
    half = [idd.upper_half_array(p, u) for p, u in zip(h.patches, states)]
    g = sk.Grid(len(hh.levels), hh.dx0, hh.patches, sk.Params(zsym=1, precision=precision),
                stream=torch.cuda.Stream())
    for i, u in enumerate(half):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(hh, half, oracle.Params(), courant=0.5, zsym=True)
    g.level_step(0)
    bo.level_step(0)
    for i in range(len(hh.patches)):
        v = g.download_fields(i)
        if precision == 0:
            e = rel_err(v, bo.current(i), active_only=True)
            assert e.max() <= 1e-10, (i, e.max())
        else:
            e = _change_err(v, bo.current(i), half[i])
            assert e.max() <= 1e-4, (i, e.max())


def test_hierarchy_half_domain_equals_full_domain():
    h, states, hh = _hierarchy()
    full = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(), stream=torch.cuda.Stream())
    half = sk.Grid(len(hh.levels), hh.dx0, hh.patches, sk.Params(zsym=1), stream=torch.cuda.Stream())
    for i, (p, u) in enumerate(zip(h.patches, states)):
        full.upload_fields(i, u)
        half.upload_fields(i, idd.upper_half_array(p, u))
    for _ in range(2):
        full.level_step(0)
        half.level_step(0)
    for i, p in enumerate(h.patches):
        a = idd.upper_half_array(p, full.download_fields(i))
        e = rel_err(half.download_fields(i), a, active_only=True)
        assert e.max() <= 1e-10, (i, e.max())


def test_zsym_rejected_with_periodic_ghosts():
    ph = idd.upper_half(idd.centred_patch(16, 0.5))
    with pytest.raises(sk.SacrakError):
        sk.Grid(1, ph.dx, [ph], sk.Params(zsym=1, bc=1))
