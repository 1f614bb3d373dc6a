"""Pins of the matter-sector oracle (oracle/grhd.py; Sec. 2.1.2, 2.2):

* the hybrid EOS: continuity of the piecewise polytrope, the first law of
  the cold curve, the sound speed against finite differences, the ideal-gas
  limit;
* the conserved variables against the special-relativistic textbook forms
  in flat space, and the primitive recovery (Newton-Raphson on w) as the
  inverse of the conserved map on generic states and metrics;
* the matter terms of the Z4c right-hand side and of the constraints: on
  generic smooth metric and fluid data they converge at 4th order to the
  ADM equations with the perfect-fluid stress-energy tensor, computed by
  the independent continuum route (tests/continuum.py);
* the finite-volume scheme: a constant state is stationary exactly; a
  density wave advected with uniform velocity and pressure converges to the
  translated profile; a TOV star (tests/tov.py) is in hydrostatic and
  Einstein equilibrium to truncation order, with the Z4c + matter
  right-hand side vanishing at 4th order inside the star."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import initial_data as idd
import oracle
from oracle import grhd

from tests import continuum as C


def _flat_state(p):
    return idd.minkowski(p)


# ------------------------------------------------------------------ EOS

def test_piecewise_polytrope_continuous_and_first_law():
    eos = grhd.EOS(K0=1.0e2, gammas=[1.6, 2.5, 3.0], rho_bounds=[5e-4, 1.5e-3], gamma_th=1.8)
    for rb in eos.rho_bounds:
        lo, hi = eos.cold(rb * (1 - 1e-12)), eos.cold(rb * (1 + 1e-12))
        assert abs(lo[0] - hi[0]) <= 1e-10 * abs(lo[0])
        assert abs(lo[1] - hi[1]) <= 1e-10 * abs(lo[1])
    rho = np.array([1e-5, 3e-4, 8e-4, 1.2e-3, 2e-3, 4e-3])
    d = 1e-6 * rho
    P, e, dP = eos.cold(rho)
    de = (eos.cold(rho + d)[1] - eos.cold(rho - d)[1]) / (2 * d)
    np.testing.assert_allclose(de, P / rho ** 2, rtol=1e-7)          # d eps = P / rho^2 d rho
    dPn = (eos.cold(rho + d)[0] - eos.cold(rho - d)[0]) / (2 * d)
    np.testing.assert_allclose(dP, dPn, rtol=1e-7)


def test_sound_speed_against_finite_differences():
    eos = grhd.EOS(K0=1.0e2, gammas=[2.0], gamma_th=1.8)
    rho = np.array([1e-4, 6e-4, 1.3e-3])
    eps = eos.cold(rho)[1] * np.array([1.0, 1.5, 3.0])
    h = 1e-6
    chi = (eos.pressure(rho * (1 + h), eps) - eos.pressure(rho * (1 - h), eps)) / (2 * h * rho)
    kap = (eos.pressure(rho, eps * (1 + h)) - eos.pressure(rho, eps * (1 - h))) / (2 * h * eps)
    P = eos.pressure(rho, eps)
    hh = 1 + eps + P / rho
    np.testing.assert_allclose(eos.cs2(rho, eps), (chi + P / rho ** 2 * kap) / hh, rtol=1e-7)
    ideal = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)  # P = (G-1) rho eps
    np.testing.assert_allclose(ideal.pressure(rho, eps), (2.0 / 3.0) * rho * eps, rtol=1e-15)
    # ideal gas: cs^2 = G P / (rho h)
    Pi = ideal.pressure(rho, eps)
    np.testing.assert_allclose(ideal.cs2(rho, eps), (5.0 / 3.0) * Pi / (rho * (1 + eps + Pi / rho)), rtol=1e-13)


# ------------------------------------------------------------------ prim <-> con

def test_conserved_variables_special_relativistic_limit():
    """Flat space: D = rho W, S_i = rho h W^2 v_i, E = rho h W^2 - P with
    v_i = u_i / W, W = 1/sqrt(1 - v^2)."""
    p = idd.centred_patch(4, 1.0)
    u = _flat_state(p)
    eos = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
    rng = np.random.default_rng(5)
    shp = p.shape[1:]
    rho = 1e-3 * (1 + rng.random(shp))
    eps = eos.cold(rho)[1] * (1 + rng.random(shp))
    v = 0.6 * (rng.random((3,) + shp) - 0.5)
    W = 1 / np.sqrt(1 - (v * v).sum(axis=0))
    prim = np.concatenate([rho[None], eps[None], W[None] * v])
    cons, w, h, P = grhd.prim2con(prim, grhd.metric(u), eos)
    np.testing.assert_allclose(w, W, rtol=1e-14)
    np.testing.assert_allclose(cons[0], rho * W, rtol=1e-14)
    np.testing.assert_allclose(cons[1:4], rho * h * W ** 2 * v, rtol=1e-13)
    np.testing.assert_allclose(cons[4], rho * h * W ** 2 - P, rtol=1e-13)


def _random_states(eos, vmax, rho_max, seed):
    p, _, u = C.patch_state(16)
    rng = np.random.default_rng(seed)
    shp = p.shape[1:]
    rho = 10 ** rng.uniform(-8, math.log10(rho_max), shp)
    eps = eos.cold(rho)[1] * (1 + 2 * rng.random(shp))
    m = grhd.metric(u)
    # u_i with |v| <= vmax in the Eulerian frame: gamma^ij u_i u_j = W^2 - 1
    dirs = rng.normal(size=(3,) + shp)
    dirs /= np.sqrt((dirs * grhd._raise(m["g_uu"], dirs)).sum(axis=0))[None]
    vv = vmax * rng.random(shp)
    W = 1 / np.sqrt(1 - vv ** 2)
    ul = np.sqrt(W ** 2 - 1)[None] * dirs
    prim = np.concatenate([rho[None], eps[None], ul])
    cons, w, _, _ = grhd.prim2con(prim, m, eos)
    assert np.allclose(w, W, rtol=1e-12)
    return m, prim, cons, W, rng


def _check_back(back, ok, prim, W):
    assert ok.all()
    np.testing.assert_allclose(back[0], prim[0], rtol=1e-11)
    # eps = h - 1 - P/rho cancels to eps_mach W^2 in absolute terms
    np.testing.assert_allclose(back[1], prim[1], rtol=1e-9, atol=1e-15 * W.max() ** 2)
    np.testing.assert_allclose(back[2:5], prim[2:5], rtol=1e-9, atol=1e-12 * np.abs(prim[2:5]).max())


@pytest.mark.parametrize("vmax", [0.3, 0.95, 0.995])
def test_recovery_inverts_the_conserved_map(vmax):
    """Random states (densities up to 1.6e-3, above nuclear; Lorentz factors
    up to 10; thermal parts up to 2x the cold energy) on the generic curved
    metric of the continuum data, single Gamma = 2 polytrope: the recovery
    from w = 1 returns the state."""
    eos = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
    m, prim, cons, W, _ = _random_states(eos, vmax, 1.6e-3, 11)
    back, ok = grhd.con2prim(cons, m, eos)
    _check_back(back, ok, prim, W)


@pytest.mark.parametrize("vmax", [0.3, 0.995])
def test_recovery_from_a_nearby_guess_two_piece_eos(vmax):
    """On a two-piece polytrope with a stiff (Gamma = 2.6) dense piece, hot
    dense states can have two physical roots of f(w); started from the
    Lorentz factor of the previous step (here the state's own, perturbed by
    up to 5%) the recovery returns the state."""
    eos = grhd.EOS(K0=100.0, gammas=[1.8, 2.6], rho_bounds=[8e-4], gamma_th=1.8)
    m, prim, cons, W, rng = _random_states(eos, vmax, 1.6e-3, 12)
    guess = W * (1 + 0.1 * (rng.random(W.shape) - 0.5))
    back, ok = grhd.con2prim(cons, m, eos, w_guess=guess)
    _check_back(back, ok, prim, W)


def test_recovery_flags_unphysical_states_and_atmosphere():
    p = idd.centred_patch(4, 1.0)
    u = _flat_state(p)
    eos = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
    m = grhd.metric(u)
    cons = np.zeros((5,) + p.shape[1:])
    cons[0] = 1e-3
    cons[4] = 1.0e-3
    cons[1] = 5e-3          # |S| > E: no physical root
    prim, ok = grhd.con2prim(cons, m, eos)
    assert not ok.any()
    floor = np.full(p.shape[1:], 1e-10)
    pr, c2, reset = grhd.recover(cons, u, eos, floor)
    assert reset.all() and np.all(pr[0] == 1e-10) and np.all(pr[2:] == 0.0)
    np.testing.assert_allclose(pr[1], eos.cold(1e-10)[1], rtol=1e-15)
    ref, _, _, _ = grhd.prim2con(pr, m, eos)
    np.testing.assert_array_equal(c2, ref)


# ------------------------------------------------------------------ coupling to Z4c

@pytest.fixture(scope="module")
def coupling_runs():
    eos = grhd.EOS(K0=C.FLUID_EOS["K"], gammas=[C.FLUID_EOS["Gamma"]], gamma_th=C.FLUID_EOS["Gamma_th"])
    out = {}
    for n in (16, 32):
        p, pts, u = C.patch_state(n)
        prim = np.ascontiguousarray(C.on_points(C.fluid_prims, pts).T.reshape((5,) + p.shape[1:]))
        s = slice(p.g, p.g + p.n[0], max(p.n[0] // 8, 1))
        z, y, x = np.meshgrid(p.axis(2)[s], p.axis(1)[s], p.axis(0)[s], indexing="ij")
        sp = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
        r = oracle.rhs(p, u, oracle.Params(sigma_ko=0.0)) + grhd.z4c_matter_rhs(prim, u, eos)
        r = r[:, s, s, s].reshape(25, -1)
        ex = C.on_points(lambda q: C.z4c_rhs_continuum(q, eta=0.36, matter=True), sp).T
        c, _ = oracle.constraints(p, u)
        dH, dM = grhd.matter_constraint_terms(prim, u, eos)
        cc = np.concatenate([(c[0] + dH)[None], c[1:] + dM])[:, s, s, s].reshape(4, -1)
        cex = C.on_points(lambda q: C.constraints_continuum(q, matter=True), sp).T
        vac = C.on_points(lambda q: C.z4c_rhs_continuum(q, eta=0.36, matter=False), sp).T
        out[n] = (r, ex, cc, cex, vac)
    return out


@pytest.mark.parametrize("f", [7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 22, 23, 24], ids=lambda f: idd.FIELD_NAMES[f])
def test_matter_terms_converge_4th_order(coupling_runs, f):
    """Khat, Theta, At, Gamt and B: the oracle's vacuum RHS plus its matter
    terms converge to the ADM equations with T^{mu nu} (the matter part is
    O(8 pi rho) ~ 1e-2 of the RHS: a wrong coefficient, sign or index of a
    matter term leaves a non-converging residual)."""
    e = []
    for n in (16, 32):
        r, ex, _, _, _ = coupling_runs[n]
        e.append(np.abs(r[f] - ex[f]).max())
    r, ex, _, _, vac = coupling_runs[32]
    scale = np.abs(ex[f]).max()
    assert np.abs(ex[f] - vac[f]).max() > 1e-3 * scale   # the matter term is visible
    assert e[1] < 2e-3 * scale and np.log2(e[0] / e[1]) > 3.5, (e, scale)


@pytest.mark.parametrize("c", range(4), ids=["H", "Mx", "My", "Mz"])
def test_matter_constraints_converge_4th_order(coupling_runs, c):
    e = []
    for n in (16, 32):
        _, _, cc, cex, _ = coupling_runs[n]
        e.append(np.abs(cc[c] - cex[c]).max())
    scale = np.abs(coupling_runs[32][3][c]).max()
    assert e[1] < 2e-3 * scale and np.log2(e[0] / e[1]) > 3.5, (e, scale)


# ------------------------------------------------------------------ finite volume

def test_constant_state_is_stationary():
    p = idd.centred_patch(10, 0.5)
    u = _flat_state(p)
    eos = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
    prim = np.zeros((5,) + p.shape[1:])
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1e-3, 0.2, 0.1, -0.05, 0.02
    r = grhd.matter_rhs(p, prim, u, eos)
    assert np.abs(r).max() <= 1e-18


def _advection_error(n, T=0.5):
    """rho = 1 + 0.2 sin(2 pi x), uniform v = 0.3 along x and P: translated."""
    dx = 1.0 / n
    p = idd.Patch(n=(n, 4, 4), dx=dx, origin=(-0.5, -2 * dx, -2 * dx))
    u = _flat_state(p)
    eos = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)
    v, P0 = 0.3, 1.0
    Wl = 1 / math.sqrt(1 - v * v)

    def prim_at(t):
        x = p.axis(0)
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * (x - v * t))
        pr = np.zeros((5,) + p.shape[1:])
        pr[0] = rho[None, None, :]
        pr[1] = P0 / ((5.0 / 3.0 - 1.0) * pr[0])
        pr[2] = Wl * v
        return pr

    m = grhd.metric(u)
    cons, _, _, _ = grhd.prim2con(prim_at(0.0), m, eos)
    floor = np.full(p.shape[1:], 1e-12)
    dt = 0.25 * dx
    steps = int(round(T / dt))
    for _ in range(steps):
        cons, pr = grhd.rk4_step_cowling(p, cons, u, dt, eos, floor, bc="periodic")
    g = p.g
    d = pr[0, g:-g, g:-g, g:-g] - prim_at(steps * dt)[0, g:-g, g:-g, g:-g]
    return np.abs(d).mean(), np.abs(d).max()


def test_density_wave_advection_converges():
    """L1 error of the translated profile falls at 2nd order or better; the
    max-norm rate is lower (about 1.4), PPM's monotonicity constraints
    clipping the smooth extrema."""
    (l32, m32), (l64, m64) = _advection_error(32), _advection_error(64)
    assert l64 < 3e-4 and math.log2(l32 / l64) > 1.8, (l32, l64)
    assert m64 < 2e-3 and m64 < m32, (m32, m64)


@pytest.fixture(scope="module")
def tov_runs():
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    out = {"star": star}
    for n in (32, 64):
        p = idd.centred_patch(n, 24.0 / n)
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        rb = np.sqrt(x * x + y * y + z * z)
        rho, psi, al = star.fields(rb)
        u = idd.minkowski(p)
        u[0] = psi ** -2
        u[18] = al
        floor = grhd.atmosphere_floor(p, 1.28e-3)
        prim = np.zeros((5,) + p.shape[1:])
        prim[0] = np.maximum(rho, floor)
        prim[1] = eos.cold(prim[0])[1]
        r_m = grhd.matter_rhs(p, prim, u, eos)
        r_z = oracle.rhs(p, u, oracle.Params(sigma_ko=0.0)) + grhd.z4c_matter_rhs(prim, u, eos)
        c, _ = oracle.constraints(p, u)
        dH, _ = grhd.matter_constraint_terms(prim, u, eos)
        out[n] = (p, rb, r_m, r_z, c[0] + dH, u, prim)
    return out


def _shell(p, rb, a):
    g = p.g
    sl = (slice(g, -g),) * 3
    m = (rb[sl] > 2.0) & (rb[sl] < 6.0)
    return a[(Ellipsis,) + sl][..., m]


def test_tov_hydrostatic_equilibrium(tov_runs):
    """Inside the star the pressure gradient balances gravity: the matter
    right-hand side (flux divergence + sources) vanishes to truncation
    order, 2nd order in the shell 2 < rbar < 6 (R = 8.1) averaged over the
    shell (L1; every axis line tangent to a sphere has a 1D extremum of rho
    there, where PPM clips its parabola, so the max-norm falls at 1st
    order)."""
    e = {}
    for n in (32, 64):
        p, rb, r_m, _, _, _, _ = tov_runs[n]
        e[n] = [np.abs(_shell(p, rb, r_m[k])).mean() for k in range(5)]
    p, rb, r_m, _, _, u, prim = tov_runs[64]
    # the scale of each balancing term: sqrt(gamma) (rho_H + P) d_i ln alpha
    scale = np.abs(_shell(p, rb, prim[0] * np.gradient(np.log(u[18]), p.dx, axis=2))).max()
    for k in range(5):
        assert e[64][k] < 2e-2 * scale and math.log2(e[32][k] / e[64][k]) > 1.6, (k, e, scale)


def test_tov_einstein_equilibrium(tov_runs):
    """The static star solves the Einstein equations: inside it the Z4c right-
    hand side with the matter terms vanishes at 4th order (Khat, Theta, At
    carry the matter terms; the others vanish exactly), and so does H."""
    for f in range(25):
        p, rb, _, r_z, _, _, _ = tov_runs[32]
        if f not in (7, 8, 9, 10, 11, 12, 13, 14):
            assert np.abs(_shell(p, rb, r_z[f])).max() == 0.0, f
    for f in (7, 8, 9, 12, 14):  # Khat, Theta, At_xx, At_yy, At_zz
        e = [np.abs(_shell(tov_runs[n][0], tov_runs[n][1], tov_runs[n][3][f])).max() for n in (32, 64)]
        assert math.log2(e[0] / e[1]) > 3.5, (f, e)
    e = [np.abs(_shell(tov_runs[n][0], tov_runs[n][1], tov_runs[n][4])).max() for n in (32, 64)]
    assert math.log2(e[0] / e[1]) > 3.5, e
    # the matter term is what balances: without it Khat's RHS is O(4 pi alpha rho)
    p, rb, _, r_z, _, u, prim = tov_runs[64]
    vac = oracle.rhs(p, u, oracle.Params(sigma_ko=0.0))[7]
    assert np.abs(_shell(p, rb, vac)).max() > 100 * np.abs(_shell(p, rb, r_z[7])).max()


def test_characteristic_speeds_closed_form():
    """Conformally flat metric (gamma_ij = delta_ij), lapse alpha and shift
    beta^x: for motion along x the fastest speeds of the HLLE flux are the
    special-relativistic velocity additions of the sound speed, alpha (v +-
    c_s) / (1 +- v c_s) - beta^x."""
    p = idd.centred_patch(4, 1.0)
    u = idd.minkowski(p)
    u[18] = 0.7
    u[19] = 0.1
    eos = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = 1e-3
    prim[1] = 0.15
    v = 0.6
    prim[2] = v / math.sqrt(1 - v * v)
    m = grhd.metric(u)
    _, _, lp, lm = grhd._flux(prim, m, eos, 0)
    cs = np.sqrt(eos.cs2(prim[0], prim[1]))
    np.testing.assert_allclose(lp, 0.7 * (v + cs) / (1 + v * cs) - 0.1, rtol=1e-13)
    np.testing.assert_allclose(lm, 0.7 * (v - cs) / (1 - v * cs) - 0.1, rtol=1e-13)
