"""Pins of the oracle against closed forms and exact special cases:
Minkowski, Brill-Lindquist puncture data, the gauge wave, the Sommerfeld
outgoing wave, the algebraic constraints, the periodic ghost fill and the
pi symmetry (Sec. 2.1.1, 2.2, 2.2.2, 3.2)."""
import math

import numpy as np
import pytest

import initial_data as idd
import oracle


def _act(p, a):
    g = p.g
    return a[..., g:-g, g:-g, g:-g]


# ------------------------------------------------------------------ Minkowski

@pytest.mark.parametrize("terms", [1, 2, 4, 7])
def test_minkowski_rhs_is_exactly_zero(terms):
    p = idd.centred_patch(12, 0.5)
    u = idd.minkowski(p)
    r = oracle.rhs(p, u, oracle.Params(), terms=terms)
    assert np.all(r == 0.0)
    assert np.all(oracle.sommerfeld_rhs(p, u) == 0.0)


def test_minkowski_rk4_step_is_exact():
    p = idd.centred_patch(10, 0.5)
    u = idd.minkowski(p)
    u1 = oracle.rk4_step(p, u, 0.25, oracle.Params())
    assert np.array_equal(u, u1)


# ------------------------------------------------------------------ Brill-Lindquist

def _bl(n, half=4.0, m=1.0):
    p = idd.single_puncture_patch(n, half)
    return p, idd.punctures(p, [m], [(0.0, 0.0, 0.0)])


def test_puncture_first_rhs_vanishing_fields():
    """K = At = beta = 0 and gt = delta: the RHS of W, alpha, gt, Gamt, beta, B
    vanish exactly (sigma_KO = 0), and Theta's RHS equals alpha H / 2."""
    p, u = _bl(16)
    prm = oracle.Params(sigma_ko=0.0)
    r = _act(p, oracle.rhs(p, u, prm))
    for f in [0, 1, 2, 3, 4, 5, 6, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24]:
        assert np.all(r[f] == 0.0), idd.FIELD_NAMES[f]
    c, _ = oracle.constraints(p, u)
    np.testing.assert_allclose(r[8], 0.5 * _act(p, u)[18] * _act(p, c)[0], rtol=1e-12, atol=1e-14)
    # momentum constraint vanishes exactly (At = K = 0)
    assert np.all(_act(p, c)[1:] == 0.0)


def test_puncture_khat_rhs_converges_to_closed_form():
    """For psi = 1 + m/(2r), alpha = W = psi^-2, flat gt: d_t Khat = -D^i D_i alpha
    = -2 psi^-8 |grad psi|^2 (Laplacian of the conformally flat metric with
    grad^2 psi = 0).  Compared on the shell 2 <= r <= 3.5 at 4th order."""
    errs = []
    for n in (16, 32):
        p, u = _bl(n)
        r = _act(p, oracle.rhs(p, u, oracle.Params(sigma_ko=0.0)))[7]
        g = p.g
        z, y, x = np.meshgrid(p.axis(2)[g:-g], p.axis(1)[g:-g], p.axis(0)[g:-g], indexing="ij")
        rr = np.sqrt(x * x + y * y + z * z)
        psi = 1.0 + 0.5 / rr
        dpsi = 0.5 / rr ** 2
        ex = -2.0 * psi ** -8 * dpsi ** 2
        m = (rr > 2.0) & (rr < 3.5)
        errs.append(np.abs(r[m] - ex[m]).max())
    rate = math.log2(errs[0] / errs[1])
    assert rate > 3.5, (errs, rate)


def test_puncture_hamiltonian_constraint_converges():
    """Brill-Lindquist data solves H = 0 exactly; the discrete H converges to 0 at
    4th order away from the puncture (Sec. 2.3)."""
    errs = []
    for n in (16, 32):
        p, u = _bl(n)
        c, _ = oracle.constraints(p, u)
        g = p.g
        z, y, x = np.meshgrid(p.axis(2)[g:-g], p.axis(1)[g:-g], p.axis(0)[g:-g], indexing="ij")
        rr = np.sqrt(x * x + y * y + z * z)
        m = (rr > 2.0) & (rr < 3.5)
        errs.append(np.abs(_act(p, c)[0][m]).max())
    assert math.log2(errs[0] / errs[1]) > 3.5, errs


def test_lapse_source_choice():
    """1+log slicing with K = Khat + 2 Theta (literal reading of Sec. 2.1.1)
    versus the Khat variant: they differ by -4 alpha Theta."""
    p = idd.centred_patch(8, 0.5)
    u = idd.minkowski(p)
    u[8] = 0.01
    a = _act(p, oracle.rhs(p, u, oracle.Params(sigma_ko=0.0)))[18]
    b = _act(p, oracle.rhs(p, u, oracle.Params(sigma_ko=0.0, lapse_uses_khat=1)))[18]
    np.testing.assert_allclose(a - b, -4.0 * 0.01, rtol=1e-14)


# ------------------------------------------------------------------ gauge wave

def _gw_patch(n):
    # quasi 1D: n cells along x, 4 along y and z, periodic box of length 1
    dx = 1.0 / n
    return idd.Patch(n=(n, 4, 4), dx=dx, origin=(-0.5, -2 * dx, -2 * dx))


def _gw_error(n, T, amp=0.01, courant=0.25):
    p = _gw_patch(n)
    prm = oracle.Params(lapse=1, shift=1, sigma_ko=0.0, kappa1=0.0)
    u = oracle.fill_periodic(p, idd.gauge_wave(p, amp))
    dt = courant * p.dx
    steps = int(round(T / dt))
    for _ in range(steps):
        u = oracle.rk4_step(p, u, dt, prm, bc=oracle.BC_PERIODIC)
    ex = idd.gauge_wave(p, amp, t=steps * dt)
    return np.abs(_act(p, u) - _act(p, ex)).max()


def test_gauge_wave_rhs_is_time_derivative():
    """At t = 0 the RHS equals d/dt of the closed-form solution (4th order);
    the time derivative is taken by a centred difference of the closed form
    with a tiny step."""
    errs = []
    for n in (16, 32):
        p = _gw_patch(n)
        prm = oracle.Params(lapse=1, shift=1, sigma_ko=0.0, kappa1=0.0)
        u = idd.gauge_wave(p, 0.01)
        r = _act(p, oracle.rhs(p, u, prm))
        eps = 1e-5
        dudt = (idd.gauge_wave(p, 0.01, t=eps) - idd.gauge_wave(p, 0.01, t=-eps)) / (2 * eps)
        errs.append(np.abs(r - _act(p, dudt)).max())
    assert errs[1] < 1e-4 and math.log2(errs[0] / errs[1]) > 3.5, errs


def test_gauge_wave_evolution_converges_4th_order():
    """RK4 + periodic ghosts + the Z4c RHS evolve the gauge wave (harmonic
    slicing, zero shift) with 4th-order global error."""
    e = [_gw_error(n, 0.25) for n in (16, 32)]
    assert math.log2(e[0] / e[1]) > 3.5, e


# ------------------------------------------------------------------ outer boundary

def test_sommerfeld_outgoing_wave():
    """For f = 1 + F(t - r)/r the condition d_t(r f) + d_r(r f) = 0 holds exactly;
    the discrete ghost RHS converges to d_t f = F'(-r)/r at 2nd order (the
    one-sided differences are 2nd order)."""
    errs = []
    for n in (16, 32):
        p = idd.single_puncture_patch(n, 4.0)
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        r = np.sqrt(x * x + y * y + z * z)
        F = lambda s: np.exp(-((s + 4.0) ** 2) / 4.0)
        dF = lambda s: -(s + 4.0) / 2.0 * F(s)
        u = idd.minkowski(p)
        u[0] = 1.0 + F(-r) / r
        u[9] = F(-r) / r
        rhs = oracle.sommerfeld_rhs(p, u)
        ghost = np.ones(r.shape, bool)
        ghost[p.g:-p.g, p.g:-p.g, p.g:-p.g] = False
        ex = dF(-r) / r
        errs.append(max(np.abs(rhs[0][ghost] - ex[ghost]).max(), np.abs(rhs[9][ghost] - ex[ghost]).max()))
        assert np.all(_act(p, rhs) == 0.0)
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_periodic_fill_brute_force():
    p = idd.Patch(n=(5, 6, 7), dx=0.1, origin=(0.0, 0.0, 0.0))
    rng = np.random.default_rng(1)
    u = rng.standard_normal(p.shape)
    v = oracle.fill_periodic(p, u)
    g = p.g
    for (k, j, i) in [(0, 0, 0), (1, 4, 10), (12, 11, 2), (5, 2, 1), (9, 8, 7)]:
        si = g + (i - g) % 5
        sj = g + (j - g) % 6
        sk = g + (k - g) % 7
        assert np.array_equal(v[:, k, j, i], u[:, sk, sj, si])


# ------------------------------------------------------------------ algebraic constraints

def test_enforcement_unit_determinant_and_trace_free():
    p = idd.centred_patch(6, 0.5)
    rng = np.random.default_rng(3)
    u = idd.minkowski(p)
    for a in range(6):
        u[1 + a] += 0.05 * rng.standard_normal(u[0].shape)
        u[9 + a] = 0.1 * rng.standard_normal(u[0].shape)
    u[0] = 1e-12  # below the floor
    v = oracle.enforce(p, u, w_floor=1e-10, all_points=True)
    g = v[1:7]
    det = (g[0] * (g[3] * g[5] - g[4] ** 2) - g[1] * (g[1] * g[5] - g[4] * g[2])
           + g[2] * (g[1] * g[4] - g[3] * g[2]))
    np.testing.assert_allclose(det, 1.0, atol=1e-14)
    M = np.array([[g[0], g[1], g[2]], [g[1], g[3], g[4]], [g[2], g[4], g[5]]]).transpose(2, 3, 4, 0, 1)
    Mi = np.linalg.inv(M)
    A = v[9:15]
    Am = np.array([[A[0], A[1], A[2]], [A[1], A[3], A[4]], [A[2], A[4], A[5]]]).transpose(2, 3, 4, 0, 1)
    tr = np.einsum("...ij,...ij->...", Mi, Am)
    np.testing.assert_allclose(tr, 0.0, atol=1e-14)
    assert np.all(v[0] == 1e-10)
    # the conformal metric direction is unchanged (pure rescaling)
    np.testing.assert_allclose(v[2] / v[1], u[2] / u[1], rtol=1e-14)


# ------------------------------------------------------------------ pi symmetry (Sec. 3.2)

def test_pi_symmetrised_data_is_symmetric_and_noise_is_not():
    p = idd.single_puncture_patch(16)
    u = idd.single_puncture_data(p, pi_symmetric=False)
    assert oracle.pi_symmetry(p, u) > 0.0
    us = idd.single_puncture_data(p, pi_symmetric=True)
    assert oracle.pi_symmetry(p, us) == 0.0


def test_pi_symmetry_of_rhs_and_rk4_bitwise():
    """Symmetrised noisy puncture data stays pi symmetric to the last bit
    through the RHS (all terms, incl. both upwind branches: the noise makes the
    shift change sign) and through RK4 steps with Sommerfeld ghosts."""
    p = idd.single_puncture_patch(16)
    u = idd.single_puncture_data(p, noise=1e-6, pi_symmetric=True)
    prm = oracle.Params()
    r = oracle.rhs(p, u, prm)
    assert oracle.pi_symmetry(p, r) == 0.0
    assert np.abs(r).max() > 0.0
    v = u
    for _ in range(2):
        v = oracle.rk4_step(p, v, 0.5 * p.dx, prm)
        assert oracle.pi_symmetry(p, v) == 0.0
    assert not np.array_equal(u, v)


def test_pi_symmetry_binary_rk4_bitwise():
    p = idd.centred_patch(16, 0.75)
    u = idd.punctures(p, [0.5, 0.5], [(2.0, 0.0, 0.0), (-2.0, 0.0, 0.0)])
    u = idd.symmetrise_pi(p, idd.add_noise(p, u, 1e-8, 7))
    v = oracle.rk4_step(p, u, 0.5 * p.dx, oracle.Params())
    assert oracle.pi_symmetry(p, v) == 0.0
