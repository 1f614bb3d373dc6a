"""TMA-staged mixed-precision stage kernels (tile shapes 32x4x1, 32x2x2,
32x4x2, 32x8x1), the L1-path, split and two-points-per-thread kernels, and
the autotuner, through the C ABI.

Every kernel is held to the mixed path's tolerances against the FP64 oracle
(1e-4 of each field's RHS scale, 1e-4 of the change an RK4 step makes), and
to the direct mixed kernel (the two differ by FP32 rounding order only:
2e-5 of the RHS scale).  pi symmetry stays bitwise (Sec. 3.2)."""
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

TMA = [1, 2, 3, 4]
# L1 path, split launches and two points per thread with 128-bit loads: the
# same arithmetic
PAIRS = [5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20]
TOL = 1e-4          # mixed precision vs the FP64 oracle
TOL_KERNELS = 2e-5  # TMA kernel vs direct mixed kernel, same data


def _change_err(v, vo, u0, g=3):
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    d = np.abs(v[a] - vo[a]).max(axis=(1, 2, 3))
    s = np.abs(vo[a] - u0[a]).max(axis=(1, 2, 3))
    return np.where(s > 0, d / np.where(s > 0, s, 1.0), d)


def _rhs(p, u, kernel, **prm):
    g = grid_for([p], precision=1, **prm)
    g.set_stage_kernel(0, kernel)
    assert g.stage_kernel(0) == kernel
    g.upload_fields(0, u)
    r = g.rhs(0)
    g.close()
    return r


@pytest.mark.parametrize("kernel", TMA + PAIRS)
def test_tma_rhs_puncture(kernel):
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    r = _rhs(p, u, kernel)
    ro = oracle.rhs(p, u, oracle.Params())
    e = rel_err(r, ro)
    assert e.max() <= TOL, dict(zip(idd.FIELD_NAMES, e))
    e0 = rel_err(r, _rhs(p, u, 0))
    assert e0.max() <= TOL_KERNELS, dict(zip(idd.FIELD_NAMES, e0))


@pytest.mark.parametrize("kernel", TMA + PAIRS)
@pytest.mark.parametrize("n", [(40, 10, 7), (33, 9, 5), (64, 12, 4)])
def test_tma_ragged_patch_rhs(kernel, n):
    """Tiles cut by the patch edge in x, y and z: the copies past the array
    are filled with zeros and the points beyond the patch write nothing."""
    ty, tz = {1: (4, 1), 2: (2, 2), 3: (4, 2), 4: (8, 1)}.get(kernel, (1, 1))
    if n[1] < ty or n[2] < tz:
        pytest.skip("patch thinner than the tile")
    dx = 0.25
    p = idd.Patch(n=n, dx=dx, origin=tuple(-0.5 * m * dx + 0.3 for m in n))
    u = idd.add_noise(p, idd.punctures(p, [0.7], [(0.1, -0.2, 0.05)]), 1e-6, 11)
    u[19:22] += 0.05 * np.sin(np.arange(u[0].size).reshape(u[0].shape) * 0.001)[None]
    r = _rhs(p, u, kernel)
    ro = oracle.rhs(p, u, oracle.Params())
    assert rel_err(r, ro).max() <= TOL
    r0 = _rhs(p, u, 0)
    assert rel_err(r, r0).max() <= TOL_KERNELS
    # ghost entries of the output stay zero
    g = 3
    inner = np.zeros(r.shape, bool)
    inner[:, g:-g, g:-g, g:-g] = True
    assert np.all(r[~inner] == 0.0)


@pytest.mark.parametrize("kernel", TMA + PAIRS)
def test_tma_rhs_gauge_wave(kernel):
    p = idd.Patch(n=(32, 4, 4), dx=1 / 32, origin=(-0.5, -2 / 32, -2 / 32))
    if kernel == 4:
        pytest.skip("patch thinner than the tile (8 rows)")
    u = oracle.fill_periodic(p, idd.gauge_wave(p, 0.01))
    r = _rhs(p, u, kernel, lapse=1, shift=1, bc=1, courant=0.25)
    ro = oracle.rhs(p, u, oracle.Params(lapse=1, shift=1))
    e = rel_err(r, ro, floor=1e-3)
    assert e.max() <= TOL, dict(zip(idd.FIELD_NAMES, e))


@pytest.mark.parametrize("kernel", [0] + TMA + PAIRS)
def test_tma_rk4_step_puncture(kernel):
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    g = grid_for([p], precision=1)
    g.set_stage_kernel(0, kernel)
    g.upload_fields(0, u)
    dt = 0.5 * p.dx
    g.rk4_step(0, dt)
    v = g.download_fields(0)
    vo = oracle.rk4_step(p, u, dt, oracle.Params())
    e = _change_err(v, vo, u)
    assert e.max() <= TOL, dict(zip(idd.FIELD_NAMES, e))


@pytest.mark.parametrize("kernel", [0] + TMA + PAIRS)
def test_tma_pi_symmetry_bitwise(kernel):
    p = idd.single_puncture_patch(32, 8.0)
    g = grid_for([p], precision=1)
    g.set_stage_kernel(0, kernel)
    g.set_initial_data(1, [1.0], [(0.0, 0.0, 0.0)], noise_amp=1e-6, seed=idd.PUNCTURE_SEED, symmetrise_pi=True)
    for _ in range(3):
        g.rk4_step(0)
        assert g.pi_symmetry(0) == 0.0


def _tma_hierarchy():
    # 3 levels, n >= 32 everywhere so that the TMA kernels run on every level;
    # the two finest patches overlap (same-level exchange is exercised)
    h = idd.small_binary(n_fixed=40, n_moving=32, n_levels=3, n_fixed_levels=2, dx0=1.0, sep=2.0)
    return h, idd.hierarchy_data(h, noise=1e-10)


@pytest.mark.parametrize("kernel", [1, 7, 10, 15, 16, 18, 19, 20])
def test_tma_level_step_hierarchy_vs_oracle(kernel):
    h, states = _tma_hierarchy()
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=1), stream=torch.cuda.Stream())
    assert all(g.stage_kernel(l) == 20 for l in range(len(h.levels)))  # the mixed-precision default
    for l in range(len(h.levels)):
        g.set_stage_kernel(l, kernel)
    for i, u in enumerate(states):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    g.level_step(0)  # recorded as a CUDA graph
    bo.level_step(0)
    for i in range(len(h.patches)):
        e = _change_err(g.download_fields(i), bo.current(i), states[i])
        assert e.max() <= TOL, (i, dict(zip(idd.FIELD_NAMES, e)))


def test_autotune_choice_and_parity():
    """The autotuner times every usable kernel per level, keeps the fastest
    (the current kernel unless another is more than 2% faster), leaves the
    state untouched, and the tuned coarse step agrees with the
    direct kernel's to FP32 rounding."""
    h, states = _tma_hierarchy()
    a = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=1), stream=torch.cuda.Stream())
    b = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=1), stream=torch.cuda.Stream())
    for i, u in enumerate(states):
        a.upload_fields(i, u)
        b.upload_fields(i, u)
    us = a.autotune(reps=2, use_cache=False)
    assert us.shape == (len(h.levels), len(sk.STAGE_KERNELS))
    for l in range(len(h.levels)):
        k = a.stage_kernel(l)
        m = us[l][us[l] > 0].min()
        # the fastest, or the level's previous kernel (20) within 2% of it
        assert us[l, k] > 0 and (us[l, k] == m or (k == 20 and m >= 0.98 * us[l, k])), (l, k, us[l])
        b.set_stage_kernel(l, 0)
    for i, u in enumerate(states):  # tuning did not touch the current level
        assert np.array_equal(a.download_fields(i), u)
    a.level_step(0)
    b.level_step(0)
    for i in range(len(h.patches)):
        va, vb = a.download_fields(i), b.download_fields(i)
        e = _change_err(va, vb, states[i])
        assert e.max() <= 1e-4, (i, e.max())
    # a second grid of the same shape takes the cached choice without timing
    c = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=1), stream=torch.cuda.Stream())
    us2 = c.autotune(reps=2, use_cache=True)
    assert np.all(us2 == -1.0)
    assert [c.stage_kernel(l) for l in range(len(h.levels))] == [a.stage_kernel(l) for l in range(len(h.levels))]


def test_tma_kernel_rejected_where_it_does_not_fit():
    p = idd.Patch(n=(24, 8, 8), dx=0.25, origin=(-3.0, -1.0, -1.0))
    g = grid_for([p], precision=1)
    assert g.stage_kernel(0) == 20
    with pytest.raises(sk.SacrakError):
        g.set_stage_kernel(0, 1)
    with pytest.raises(sk.SacrakError):
        g.set_stage_kernel(0, len(sk.STAGE_KERNELS))
    f = grid_for([idd.single_puncture_patch(32, 8.0)])  # FP64: only the direct kernel
    assert f.stage_kernel(0) == 0
    for k in (1, 5, 15):
        with pytest.raises(sk.SacrakError):
            f.set_stage_kernel(0, k)


@pytest.mark.parametrize("n", [(32, 32, 20), (48, 48, 9), (64, 64, 5), (96, 96, 4), (40, 32, 6)])
def test_fixed_pitch_kernel_is_kernel_10_bitwise(n):
    """Kernels 19 and 20 (the pitches of patches n[0] = n[1] in {32, 48, 64,
    96, ...} fixed at compile time, 3 and 4 CTAs per SM; (40, 32) has no
    instance and runs kernel 10): two RK4 steps give kernel 10's state bit
    for bit."""
    dx = 0.25
    p = idd.Patch(n=n, dx=dx, origin=tuple(-0.5 * m * dx + 0.3 for m in n))
    u = idd.add_noise(p, idd.punctures(p, [0.7], [(0.1, -0.2, 0.05)]), 1e-6, 11)
    u[19:22] += 0.05 * np.sin(np.arange(u[0].size).reshape(u[0].shape) * 0.001)[None]
    out = {}
    for kernel in (10, 19, 20):
        g = grid_for([p], precision=1)
        g.set_stage_kernel(0, kernel)
        g.upload_fields(0, u)
        for _ in range(2):
            g.rk4_step(0, 0.25 * dx)
        out[kernel] = g.download_fields(0)
    assert np.array_equal(out[10], out[19]) and np.array_equal(out[10], out[20])
    assert np.abs(out[19] - u).max() > 0.0
