"""Pins of the oracle's face flux (Sec. 2.2): the HLLC flux of special
relativity solved in an orthonormal tetrad in which the face is at rest,
with the HLLE flux there where the intermediate state is unphysical
(oracle/grhd.py: face_tetrad, sr_hllc, hllc_tetrad_flux).

* The tetrad is orthonormal in the face metric, e0, e2, e3 are tangent to
  the face's world-sheet (no component along x^d), and it is the coordinate
  basis in flat space.
* Equal left and right states give the physical flux of the coordinate
  frame, computed by the other route (the 3+1 fluxes of oracle/grhd._flux):
  this pins the transformation into the tetrad and back, on random metrics
  and states.
* Contacts: two states with the same four-velocity and pressure and
  different density are an isolated contact, which HLLC resolves exactly:
  the flux is the physical flux of the upwind state (the side the fluid
  comes from), in flat space and on random metrics; at rest, the mass and
  energy fluxes vanish and the momentum flux is the pressure.  HLLE smears
  the contact (non-zero mass flux at rest).
* Mirror symmetry: swapping the two states and reversing the normal
  velocity reverses the mass, transverse-momentum and energy fluxes and
  keeps the normal-momentum flux.
* Fallback: states receding from each other fast enough give a negative
  intermediate pressure; the flux is then the HLLE flux.
* A density step at rest with uniform pressure (a contact discontinuity)
  stays in place to rounding through RK4 steps of the whole scheme; with
  HLLE it spreads."""
import math

import numpy as np
import pytest

import initial_data as idd
from oracle import grhd

SYM = grhd.SYM


def _random_metric(rng, n, amp=0.2):
    al = 0.6 + 0.4 * rng.random(n)
    be = amp * (rng.random((3, n)) - 0.5)
    A = amp * rng.random((3, 3, n))
    g = np.empty((6, n))
    for c, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        g[c] = (1.0 if i == j else 0.0) + 0.5 * (A[i, j] + A[j, i])
    gu, det = grhd._inv_sym(g)
    return {"alpha": al, "beta": be, "g_ll": g, "g_uu": gu, "sqrtg": np.sqrt(det)}


def _flat_metric(n):
    g = np.zeros((6, n))
    g[0] = g[3] = g[5] = 1.0
    return {"alpha": np.ones(n), "beta": np.zeros((3, n)), "g_ll": g, "g_uu": g.copy(), "sqrtg": np.ones(n)}


EOS = grhd.EOS(K0=100.0, gammas=[2.0], gamma_th=1.8)
GAS = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)  # ideal gas, P = (5/3 - 1) rho eps


def _random_prim(rng, n, umax=0.5):
    return np.array([1e-3 * (1.0 + rng.random(n)), 0.05 * (1.0 + rng.random(n)),
                     *(umax * (rng.random((3, n)) - 0.5))])


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("d", [0, 1, 2])
def test_tetrad_orthonormal_and_tangent_to_the_face(d):
    rng = np.random.default_rng(11 + d)
    m = _random_metric(rng, 9)
    e, s1 = grhd.face_tetrad(m, d)
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    for a in range(4):
        for b in range(4):
            assert np.abs(grhd._dot4(m, e[a], e[b]) - eta[a, b]).max() <= 1e-14
    for a in (0, 2, 3):
        assert np.abs(e[a][1 + d]).max() <= 1e-15   # xi_mu e^mu = e^d = 0
    # e1 along xi = dx^d: (e1)_mu = g_{mu nu} e1^nu has only the d component
    assert np.allclose(s1 ** 2, m["g_uu"][SYM[d][d]] - m["beta"][d] ** 2 / m["alpha"] ** 2)
    ef, _ = grhd.face_tetrad(_flat_metric(3), d)
    basis = [0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3]
    for a in range(4):
        want = np.zeros((4, 3))
        want[basis[a]] = 1.0
        assert np.abs(ef[a] - want).max() <= 1e-15


@pytest.mark.parametrize("d", [0, 1, 2])
def test_equal_states_give_the_coordinate_flux(d):
    rng = np.random.default_rng(21 + d)
    m = _random_metric(rng, 12)
    prim = _random_prim(rng, 12)
    f = grhd.hllc_tetrad_flux(prim, prim, m, EOS, d)
    _, F, _, _ = grhd._flux(prim, m, EOS, d)
    assert _rel(f, F) <= 1e-13


def _contact_pair(rng, n, umax=0.5):
    """Same u_i and pressure, densities differing by a factor 1.5-3."""
    pl = _random_prim(rng, n, umax)
    pr = pl.copy()
    pr[0] = pl[0] * (1.5 + 1.5 * rng.random(n))
    P = GAS.pressure(pl[0], pl[1])
    pr[1] = P / ((GAS.gamma_th - 1.0) * pr[0])
    return pl, pr


def test_contact_at_rest_in_flat_space_is_exact():
    rng = np.random.default_rng(5)
    n = 6
    m = _flat_metric(n)
    pl, pr = _contact_pair(rng, n)
    for v in (2, 3, 4):
        pl[v] = pr[v] = 0.0
    P = GAS.pressure(pl[0], pl[1])
    f = grhd.hllc_tetrad_flux(pl, pr, m, GAS, 0)
    assert np.abs(f[[0, 2, 3, 4]]).max() <= 1e-15 * P.max()
    assert np.abs(f[1] - P).max() <= 1e-15 * P.max()
    h = grhd.hlle_flux(pl, pr, m, GAS, 0)
    assert np.abs(h[0]).min() > 1e-6 * np.abs(pl[0]).max()  # HLLE diffuses the density jump


@pytest.mark.parametrize("metric", ["flat", "random"])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_moving_contact_takes_the_upwind_flux(metric, d):
    rng = np.random.default_rng(31 + d)
    n = 16
    m = _flat_metric(n) if metric == "flat" else _random_metric(rng, n)
    pl, pr = _contact_pair(rng, n)
    f = grhd.hllc_tetrad_flux(pl, pr, m, GAS, d)
    _, FL, _, _ = grhd._flux(pl, m, GAS, d)
    _, FR, _, _ = grhd._flux(pr, m, GAS, d)
    # the contact moves with the fluid: through the face towards +d where
    # the coordinate velocity V^d = alpha u^d / w - beta^d is positive
    uu = grhd._raise(m["g_uu"], pl[2:5])
    w = np.sqrt(1.0 + (pl[2:5] * uu).sum(axis=0))
    V = m["alpha"] * uu[d] / w - m["beta"][d]
    want = np.where(V[None] > 0, FL, FR)
    assert _rel(f, want) <= 1e-12


def test_mirror_symmetry():
    rng = np.random.default_rng(41)
    n = 10
    m = _flat_metric(n)
    pl, pr = _random_prim(rng, n), _random_prim(rng, n)
    f = grhd.hllc_tetrad_flux(pl, pr, m, EOS, 0)
    ml, mr = pr.copy(), pl.copy()
    ml[2] *= -1.0
    mr[2] *= -1.0
    g = grhd.hllc_tetrad_flux(ml, mr, m, EOS, 0)
    # mirror x -> -x: D, S_y, S_z, E fluxes change sign, S_x flux does not
    sign = np.array([-1.0, 1.0, -1.0, -1.0, -1.0])[:, None]
    assert _rel(g, sign * f) <= 1e-13


def test_receding_states_fall_back_to_hlle():
    n = 3
    m = _flat_metric(n)
    e, _ = grhd.face_tetrad(m, 0)
    W = 1.0 / math.sqrt(1.0 - 0.9 ** 2)
    pl = np.array([np.ones(n), np.full(n, 1.5), np.full(n, -0.9 * W), np.zeros(n), np.zeros(n)])
    pr = pl.copy()
    pr[2] = 0.9 * W
    L = grhd._sr_state(pl, m, GAS, e)
    R = grhd._sr_state(pr, m, GAS, e)
    F, ok = grhd.sr_hllc(*L, *R)
    assert not ok.any()
    lL = np.minimum(L[3], R[3])
    lR = np.maximum(L[2], R[2])
    Fh = (lR * L[1] - lL * R[1] + lL * lR * (R[0] - L[0])) / (lR - lL)
    assert _rel(F, Fh) <= 1e-15
    # the HLL average of the receding pair has no positive contact pressure
    Uh = (lR * R[0] - lL * L[0] + L[1] - R[1]) / (lR - lL)
    Fhl = (lR * L[1] - lL * R[1] + lL * lR * (R[0] - L[0])) / (lR - lL)
    b = Uh[4] + Fhl[1]
    ls = 2.0 * Uh[1] / (b + np.sqrt(b * b - 4.0 * Fhl[4] * Uh[1]))
    assert (Fhl[1] - ls * Fhl[4] <= 0.0).all()


def _step_after(solver, n=32, steps=20):
    """A density step (square wave, densities 1 and 2) at rest with uniform
    pressure, periodic along x, after `steps` RK4 steps."""
    dx = 1.0 / n
    p = idd.Patch(n=(n, 4, 4), dx=dx, origin=(-0.5, -2 * dx, -2 * dx))
    u = idd.minkowski(p)
    pr = np.zeros((5,) + p.shape[1:])
    pr[0] = np.where(np.abs(p.axis(0)) < 0.25, 2.0, 1.0)[None, None, :]
    pr[1] = 1.0 / ((GAS.gamma_th - 1.0) * pr[0])
    cons, _, _, _ = grhd.prim2con(pr, grhd.metric(u), GAS)
    floor = np.full(p.shape[1:], 1e-12)
    for _ in range(steps):
        cons, out = grhd.rk4_step_cowling(p, cons, u, 0.25 * dx, GAS, floor, bc="periodic", solver=solver)
    g = p.g
    return np.abs(out[0, g:-g, g:-g, g:-g] - pr[0, g:-g, g:-g, g:-g]).max()


def test_contact_discontinuity_at_rest_stays_exact():
    """HLLC keeps a density step at rest in place to rounding; HLLE spreads
    it over the neighbouring cells."""
    assert _step_after("hllc") <= 1e-13
    assert _step_after("hlle") > 1e-2
