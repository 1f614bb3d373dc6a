"""Long evolutions on the GPU against what the method fixes (the
gauge-wave and robust-stability checks of the Z4c literature that the
paper's scheme is built from, Sec. 2.1.1/2.2): the gauge wave on a periodic
3D grid converges to its closed form at 4th order, and noisy Minkowski data
stays bounded.  Reduced sizes here; bench.py --case gauge-wave /
robust-stability runs the 32^3 / 64^3 / 128^3 versions."""
import math

import numpy as np
import pytest

import initial_data as idd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

skbuild.build()


def _grid(n, precision=0):
    p = idd.centred_patch(n, 1.0 / n)
    g = sk.Grid(1, p.dx, [p], sk.Params(lapse=1, shift=1, bc=1, courant=0.25, precision=precision),
                stream=torch.cuda.Stream())
    return p, g


def _gw_error(n, t_final, precision=0):
    p, g = _grid(n, precision)
    g.set_initial_data(2, gw_amp=0.01, gw_len=1.0)
    steps = int(round(t_final / (0.25 * p.dx)))
    for _ in range(steps):
        g.rk4_step(0)
    t = g.level_time(0)
    assert t == pytest.approx(t_final)
    u = g.download_fields(0)[:, 3:-3, 3:-3, 3:-3]
    ex = idd.gauge_wave(p, 0.01, t=t)[:, 3:-3, 3:-3, 3:-3]
    g.close()
    return np.abs(u - ex).max()


def test_gauge_wave_3d_converges_4th_order_fp64():
    e = [_gw_error(n, 0.5) for n in (16, 32)]
    rate = math.log2(e[0] / e[1])
    assert e[1] < 2e-5 and rate > 3.5, (e, rate)


def test_gauge_wave_3d_mixed_precision_error_near_fp64():
    """The mixed path adds FP32 rounding of the RHS (about 1e-7 relative) to
    the truncation error; at 32^3 the truncation error still dominates."""
    e64 = _gw_error(32, 0.5, 0)
    emx = _gw_error(32, 0.5, 1)
    assert abs(emx - e64) <= 0.05 * e64 + 1e-9, (e64, emx)


@pytest.mark.parametrize("precision", [0, 1])
def test_robust_stability_bounded(precision):
    """Minkowski + noise 1e-10 on every field at 32^3, 400 RK4 steps.  The
    Hamiltonian constraint decays (Kreiss-Oliger dissipation removes the
    grid-scale noise) and the momentum constraint stays bounded.  The fields
    respond to the frozen noisy shift, a constant source of grid-scale
    second derivatives in the Gamt equation, so they move away from flat
    space, but without exponential growth: over the second half of the run
    the largest deviation grows by less than the factor 2 of linear growth."""
    p, g = _grid(32, precision)
    g.set_initial_data(0, noise_amp=1e-10, seed=idd.STABILITY_SEED)
    flat = idd.minkowski(p)
    h0 = g.constraints(0)
    hist, dev = [], []
    for s in range(400):
        g.rk4_step(0)
        if (s + 1) % 100 == 0:
            hist.append(g.constraints(0))
            dev.append(np.abs(g.download_fields(0) - flat).max())
    hist = np.array(hist)
    assert np.all(np.isfinite(hist)) and np.all(np.isfinite(dev))
    assert hist[-1, 0] < h0[0], (h0, hist)
    assert hist[-1, 1:].max() <= 2.0 * hist[1, 1:].max(), hist
    assert dev[3] < 2.0 * dev[1] and dev[3] < 1e-5, dev
