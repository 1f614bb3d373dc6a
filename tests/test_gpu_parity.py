"""GPU FP64 path against the CPU oracle, element by element, through the C ABI
(tolerance 1e-12 relative max-norm per field for one RHS call and one RK4
step, Sec. 2.1.1/2.2), bitwise pi symmetry (Sec. 3.2), device initial data,
ghost treatments, ragged patch sizes and the Berger-Oliger step."""
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

TOL_RHS = 1e-12
TOL_STEP = 1e-12


def c1_patch():
    return idd.single_puncture_patch(32, 8.0)


# ------------------------------------------------------------------ initial data

def test_device_puncture_data_bitwise():
    p = c1_patch()
    g = grid_for([p])
    g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)], noise_amp=1e-10, seed=idd.PUNCTURE_SEED)
    u = g.download_fields(0)
    ref = idd.single_puncture_data(p)
    assert np.array_equal(u, ref)
    g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)], noise_amp=1e-10, seed=idd.PUNCTURE_SEED, symmetrise_pi=True)
    assert np.array_equal(g.download_fields(0), idd.single_puncture_data(p, pi_symmetric=True))
    assert g.pi_symmetry(0) == 0.0


def test_device_gauge_wave_data():
    p = idd.Patch(n=(16, 4, 4), dx=1 / 16, origin=(-0.5, -0.125, -0.125))
    g = grid_for([p], bc=1)
    g.set_initial_data(2, gw_amp=0.01, gw_len=1.0)
    np.testing.assert_allclose(g.download_fields(0), idd.gauge_wave(p, 0.01), rtol=0, atol=1e-15)


# ------------------------------------------------------------------ RHS and RK4 parity (C1)

@pytest.mark.parametrize("sym", [False, True])
def test_rhs_parity_puncture(sym):
    p = c1_patch()
    u = idd.single_puncture_data(p, pi_symmetric=sym)
    g = grid_for([p])
    g.upload_fields(0, u)
    r = g.rhs(0)
    ro = oracle.rhs(p, u, oracle.Params())
    e = rel_err(r, ro)
    assert e.max() <= TOL_RHS, dict(zip(idd.FIELD_NAMES, e))
    assert np.all(r[:, :3] == 0.0) and np.all(r[:, :, :, -3:] == 0.0)
    if sym:
        assert oracle.pi_symmetry(p, r) == 0.0


def test_rk4_step_parity_puncture_sommerfeld():
    p = c1_patch()
    u = idd.single_puncture_data(p)
    g = grid_for([p])
    g.upload_fields(0, u)
    dt = 0.5 * p.dx
    g.rk4_step(0, dt)
    v = g.download_fields(0)
    vo = oracle.rk4_step(p, u, dt, oracle.Params())
    e = rel_err(v, vo)
    assert e.max() <= TOL_STEP, dict(zip(idd.FIELD_NAMES, e))


def test_pi_symmetry_bitwise_through_steps():
    p = c1_patch()
    g = grid_for([p])
    g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)], noise_amp=1e-6, seed=idd.PUNCTURE_SEED, symmetrise_pi=True)
    assert g.pi_symmetry(0) == 0.0
    r = g.rhs(0)
    assert oracle.pi_symmetry(p, r) == 0.0
    for _ in range(3):
        g.rk4_step(0)
        assert g.pi_symmetry(0) == 0.0


def test_binary_pi_symmetry_bitwise():
    p = idd.centred_patch(32, 0.5)
    g = grid_for([p])
    g.set_initial_data(1, [0.5, 0.5], [(3.0, 0.0, 0.0), (-3.0, 0.0, 0.0)], noise_amp=1e-8, seed=5,
                       symmetrise_pi=True)
    for _ in range(2):
        g.rk4_step(0)
    assert g.pi_symmetry(0) == 0.0


# ------------------------------------------------------------------ ghosts and ragged sizes

def test_periodic_gauge_wave_steps_parity():
    p = idd.Patch(n=(32, 4, 4), dx=1 / 32, origin=(-0.5, -2 / 32, -2 / 32))
    prm = dict(lapse=1, shift=1, bc=1, sigma_ko=0.0, kappa1=0.0, courant=0.25)
    g = grid_for([p], **prm)
    u = oracle.fill_periodic(p, idd.gauge_wave(p, 0.01))
    g.upload_fields(0, u)
    op = oracle.Params(lapse=1, shift=1, sigma_ko=0.0, kappa1=0.0)
    dt = 0.25 * p.dx
    for _ in range(4):
        g.rk4_step(0, dt)
        u = oracle.rk4_step(p, u, dt, op, bc=oracle.BC_PERIODIC)
    # every non-constant field of the gauge wave is O(A) = O(0.01); fields that
    # vanish analytically (Theta) are roundoff noise, so each field is judged
    # relative to max(|field|, A)
    e = rel_err(g.download_fields(0), u, floor=0.01)
    # four RK4 steps accumulate the per-call rounding differences (1e-12 per
    # RHS call); Khat, Theta and At reach ~1e-12 relative after four steps
    assert e.max() <= 1e-11, " ".join("%s=%.2e" % kv for kv in zip(idd.FIELD_NAMES, e) if kv[1] > 1e-14)


def test_gauge_wave_rhs_parity():
    """RHS parity on the gauge wave (non-flat gt, At, K, Gamt active)."""
    p = idd.Patch(n=(32, 4, 4), dx=1 / 32, origin=(-0.5, -2 / 32, -2 / 32))
    prm = dict(lapse=1, shift=1, bc=1, sigma_ko=0.5, kappa1=0.005, courant=0.25)
    g = grid_for([p], **prm)
    u = oracle.fill_periodic(p, idd.gauge_wave(p, 0.01))
    g.upload_fields(0, u)
    r = g.rhs(0)
    ro = oracle.rhs(p, u, oracle.Params(lapse=1, shift=1, sigma_ko=0.5, kappa1=0.005))
    e = rel_err(r, ro, floor=1e-3)
    assert e.max() <= TOL_RHS, {k: "%.2e" % v for k, v in zip(idd.FIELD_NAMES, e)}


def test_frozen_ghosts_parity():
    p = idd.centred_patch(16, 0.5)
    u = idd.single_puncture_data(p, noise=1e-8)
    g = grid_for([p], bc=2)
    g.upload_fields(0, u)
    g.rk4_step(0, 0.25)
    vo = oracle.rk4_step(p, u, 0.25, oracle.Params(), bc=oracle.BC_FROZEN)
    v = g.download_fields(0)
    assert rel_err(v, vo).max() <= TOL_STEP
    gh = np.ones(v.shape[1:], bool)
    gh[3:-3, 3:-3, 3:-3] = False
    assert np.array_equal(v[:, gh], u[:, gh])


@pytest.mark.parametrize("n", [(40, 10, 6), (33, 5, 4), (7, 9, 11)])
def test_ragged_patch_rhs_parity(n):
    dx = 0.25
    p = idd.Patch(n=n, dx=dx, origin=tuple(-0.5 * m * dx + 0.3 for m in n))
    u = idd.add_noise(p, idd.punctures(p, [0.7], [(0.1, -0.2, 0.05)]), 1e-6, 11)
    u[19:22] += 0.05 * np.sin(np.arange(u[0].size).reshape(u[0].shape) * 0.001)[None]
    g = grid_for([p])
    g.upload_fields(0, u)
    r = g.rhs(0)
    ro = oracle.rhs(p, u, oracle.Params())
    assert rel_err(r, ro).max() <= TOL_RHS


def test_constraints_parity():
    p = c1_patch()
    u = idd.single_puncture_data(p)
    g = grid_for([p])
    g.upload_fields(0, u)
    n_gpu = g.constraints(0)
    _, n_orc = oracle.constraints(p, u)
    np.testing.assert_allclose(n_gpu, n_orc, rtol=1e-10, atol=1e-300)
    n_gpu = g.constraints(0, w_excise=0.3)
    _, n_orc = oracle.constraints(p, u, w_excise=0.3)
    np.testing.assert_allclose(n_gpu, n_orc, rtol=1e-10)


# ------------------------------------------------------------------ Berger-Oliger

def _small_hierarchy():
    h = idd.small_binary()
    return h, idd.hierarchy_data(h, noise=1e-10)


def test_level_step_parity_small_hierarchy():
    h, states = _small_hierarchy()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params())
    for i, u in enumerate(states):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    for step in range(2):
        g.level_step(0)
        bo.level_step(0)
        for i in range(len(h.patches)):
            e = rel_err(g.download_fields(i), bo.current(i), active_only=True)
            assert e.max() <= 1e-10, (step, i, e.max())
    assert g.level_time(len(h.levels) - 1) == pytest.approx(2 * 0.5 * h.dx0)


def test_level_step_graph_replay_matches_eager():
    """On a non-default stream level_step(0) records a CUDA graph on its first
    call and replays it; on the legacy default stream it launches eagerly.  The
    two must agree bit for bit."""
    h, states = _small_hierarchy()
    a = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(), stream=torch.cuda.Stream())
    c = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(), stream=torch.cuda.default_stream())
    for i, u in enumerate(states):
        a.upload_fields(i, u)
        c.upload_fields(i, u)
    for _ in range(3):
        a.level_step(0)
        c.level_step(0)
    for i in range(len(h.patches)):
        assert np.array_equal(a.download_fields(i), c.download_fields(i))
