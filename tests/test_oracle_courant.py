"""Linear stability of the discretisation at the Courant factor (Sec. 2.2:
4th-order centred differences, 6th-order Kreiss-Oliger dissipation with
sigma_KO = 0.5, classical RK4, Courant factor 0.5) on flat space, pinned
against a linearisation derived here by hand.

The mode is the grid's checkerboard, f_ijk = (-1)^(i+j+k), on a periodic
box: every centred first difference of it vanishes, the 4th-order second
difference D_d D_d gives -16/(3 h^2) per axis (so the discrete Laplacian is
-16/h^2), the mixed second differences vanish, and the 6th-order dissipation
sigma/(64 h) sum_d Delta_d^6 gives -3 sigma / h.  A checkerboard in the lapse
of Minkowski space (beta = B = 0, gt = delta, At = 0, Gamt = 0) therefore
stays inside (alpha, Khat, W, Theta): the trace-free parts are zero by the
symmetry of the three axes, Gamt, beta and B are driven only by first
differences.  The linearised equations (alpha = 1 + a, W = 1 + w):

* 1+log slicing (Sec. 2.1.1): a_t = -2 K with K = Khat + 2 Theta (the
  Z4c trace of K_ij), or -2 Khat where the slicing uses Khat;
* Z4c (Sec. 2.1.1, Bernuzzi & Hilditch): Khat_t = -Laplacian a
  + kappa1 (1 - kappa2) Theta, Theta_t = R / 2 - kappa1 (2 + kappa2) Theta;
* W = det(gamma)^(-1/6) with d_t gamma_ij = -2 K_ij: w_t = K / 3;
* the scalar curvature of gamma_ij = W^-2 delta_ij is 4 W Laplacian W
  - 6 |grad W|^2, so R = 4 Laplacian w to first order.

RK4 maps y -> P(dt A) y with P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 and A the
4 x 4 operator above plus the dissipation; the oracle's checkerboard
amplitudes after N steps must equal P(dt A)^N y0.  At the paper's Courant
factor the largest |eigenvalue| of P(dt A) exceeds one (4.35 per step with
K = Khat + 2 Theta in the slicing, 1.078 with Khat): the paper's Courant
factor is past the linear stability limit of this discretisation for the
gauge mode at alpha ~ 1, with a refinement boundary or without one."""
import numpy as np
import pytest

import initial_data as idd
import oracle

ALP, KH, W, TH = 18, 7, 0, 8
N = 8          # periodic 8^3 box
EPS = 1e-8     # linear regime: products of checkerboards feed only the constant mode,
               # so the checkerboard amplitude is linear up to O(EPS^2) relative


def _operator(h, khat, sigma, kappa1, kappa2=0.0):
    q = 16.0 / h ** 2                       # minus the discrete Laplacian of the checkerboard
    a_row = [0.0, -2.0, 0.0, 0.0 if khat else -4.0]
    A = np.array([a_row,
                  [q, 0.0, 0.0, kappa1 * (1.0 - kappa2)],
                  [0.0, 1.0 / 3.0, 0.0, 2.0 / 3.0],
                  [0.0, 0.0, -2.0 * q, -kappa1 * (2.0 + kappa2)]])
    return A - 3.0 * sigma / h * np.eye(4)


def _rk4_map(z):
    I = np.eye(len(z))
    return I + z + z @ z / 2 + z @ z @ z / 6 + z @ z @ z @ z / 24


def _checkerboard(p):
    i = np.arange(p.n[0] + 6)
    return (-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])


def _amplitudes(p, u, cb):
    a = (slice(3, -3),) * 3
    bg = {ALP: 1.0, KH: 0.0, W: 1.0, TH: 0.0}
    return np.array([np.mean((u[f][a] - bg[f]) * cb[a]) for f in (ALP, KH, W, TH)])


@pytest.mark.parametrize("courant,khat,sigma,kappa2", [
    (0.5, 0, 0.5, 0.0), (0.5, 1, 0.5, 0.0), (0.4, 0, 0.5, 0.0), (0.25, 0, 0.5, 0.0),
    (0.5, 0, 0.0, 0.0), (0.45, 1, 1.0, 0.0), (0.5, 0, 0.5, 0.3)])
def test_checkerboard_mode_follows_linear_rk4_map(courant, khat, sigma, kappa2):
    p = idd.centred_patch(N, 1.0 / N)
    cb = _checkerboard(p)
    u = idd.minkowski(p)
    u[ALP] += EPS * cb
    prm = oracle.Params(sigma_ko=sigma, lapse_uses_khat=khat, kappa1=0.005, kappa2=kappa2)
    dt = courant * p.dx
    M = _rk4_map(dt * _operator(p.dx, khat, sigma, 0.005, kappa2))
    y = np.array([EPS, 0.0, 0.0, 0.0])
    for _ in range(6):
        u = oracle.rk4_step(p, u, dt, prm, bc=oracle.BC_PERIODIC)
        y = M @ y
        got = _amplitudes(p, u, cb)
        # rounding: the fields are O(1), so ~1e-15 absolute per step
        np.testing.assert_allclose(got, y, rtol=0, atol=1e-7 * np.abs(y).max() + 1e-14)
    # nothing else was excited
    rest = [f for f in range(25) if f not in (ALP, KH, W, TH)]
    assert np.abs(u[rest] - idd.minkowski(p)[rest]).max() <= 1e-9 * np.abs(y).max()


def test_paper_courant_factor_is_past_the_checkerboard_limit():
    """Spectral radius of the RK4 map per step (h = 1): above one at the
    paper's Courant factor for both readings of the slicing's K, below one
    at the factor the benchmark hierarchy runs with."""
    def radius(c, khat):
        return np.abs(np.linalg.eigvals(_rk4_map(c * _operator(1.0, khat, 0.5, 0.005)))).max()
    assert radius(0.5, 0) == pytest.approx(4.354, abs=2e-3)
    assert radius(0.5, 1) == pytest.approx(1.078, abs=2e-3)
    assert radius(0.25, 0) < 1.0 and radius(0.25, 1) < 1.0
    assert radius(0.39, 0) < 1.0 < radius(0.40, 0)
    assert radius(0.49, 1) < 1.0 < radius(0.50, 1)
