"""Pins of the oracle's ADM mass and angular momentum surface integrals
(Sec. 2.3) against closed forms that do not come from the oracle itself.

* Gauss-Legendre nodes: numpy's leggauss and exact integration of
  polynomials up to degree 2n - 1.
* Schwarzschild in isotropic coordinates (one Brill-Lindquist puncture):
  gamma_ij = psi^4 delta_ij, psi = 1 + M/(2r), so the mass integrand is
  -8 psi d_i psi and M_ADM(r) = M psi(r) = M (1 + M/(2r)) on every sphere
  around the puncture; the error must fall like dx^4.
* Bowen-York spin and boost: sqrt(gamma) K_i^j = Ahat_ij for any conformal
  factor (K = 0); for spin S, Ahat_ij n^j = 3/r^3 (S x n)_i, so J_z = S_z and
  P = 0 on every sphere around the puncture; for momentum P, Ahat_ij n^j =
  3/(2 r^2) (P_i + n_i P.n), whose flux is P (and J_z = 0).
* The trace term of P^ADM: a pure-trace K_ij = K gamma_ij / 3 with
  gamma = delta gives (K/3 - K) n_i, so P_i = -(1/12 pi) int K n_i dS; for
  K = k0 + k1 x this is -(k1 r^3 / 9) e_x (int n_x^2 dOmega = 4 pi / 3; the
  k0 part cancels).
* A pure-gauge linear perturbation gamma_ij = delta_ij + eps (d_i xi_j +
  d_j xi_i) of flat space: the linearised mass integrand is the divergence of
  an antisymmetric tensor, whose flux through a closed surface vanishes, so
  M_ADM is of order eps^2 (a dropped or mis-signed term would leave an order-
  eps flux).
"""
import numpy as np
import pytest

import initial_data as idt
import oracle


def test_gauss_legendre_nodes():
    for n in (1, 2, 5, 12, 24):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        o = np.argsort(x)
        assert np.abs(x[o] - xr).max() < 1e-14
        assert np.abs(w[o] - wr).max() < 1e-14
        for k in range(2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.dot(w, x ** k) - exact) < 1e-13


def test_minkowski_zero():
    p = idt.centred_patch(32, 0.5)
    v = oracle.adm_integrals(p, idt.minkowski(p), (0.0, 0.0, 0.0), 5.0, 16, 32)
    assert v == (0.0,) * 5


def test_schwarzschild_mass_fourth_order():
    mass = 1.0
    for n in (32, 96):
        p = idt.centred_patch(n, 16.0 / n)
        u = idt.bowen_york(p, mass)
        errs = []
        for r in (4.5, 5.0, 5.5, 6.0):
            m, j, px, py, pz = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), r, 48, 96)
            errs.append(abs(m - mass * (1.0 + mass / (2.0 * r))))
            assert j == 0.0 and px == py == pz == 0.0
        # truncation C dx^4 with C measured below 3e-4 for these spheres
        assert max(errs) < 1e-3 * p.dx ** 4, (n, errs)
    # the radius dependence M psi(r) itself, not only its limit
    p = idt.centred_patch(96, 16.0 / 96)
    u = idt.bowen_york(p, 0.5)
    m4 = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), 4.0, 48, 96)[0]
    m7 = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), 7.0, 48, 96)[0]
    assert abs((m4 - m7) - 0.5 * 0.5 * (1 / 8.0 - 1 / 14.0)) < 1e-6


@pytest.mark.parametrize("spin", [(0.0, 0.0, 0.7), (0.7, 0.0, 0.0), (0.3, -0.2, 0.6)])
def test_bowen_york_spin(spin):
    p = idt.centred_patch(64, 0.25)
    c = (1.0, -0.5, 0.25)
    u = idt.bowen_york(p, 1.0, c, spin=spin)
    m, j, *P = oracle.adm_integrals(p, u, c, 5.0, 48, 96)
    assert abs(j - spin[2]) < 2e-6
    assert abs(m - 1.1) < 1e-6  # the spin does not enter the mass
    assert max(abs(v) for v in P) < 1e-6


@pytest.mark.parametrize("mom", [(0.2, 0.0, 0.0), (0.0, -0.3, 0.1), (0.1, 0.2, 0.3)])
def test_bowen_york_boost(mom):
    p = idt.centred_patch(64, 0.25)
    c = (-0.5, 0.75, 0.25)
    u = idt.bowen_york(p, 1.0, c, momentum=mom)
    for r in (4.0, 5.5):
        m, j, *P = oracle.adm_integrals(p, u, c, r, 48, 96)
        assert max(abs(a - b) for a, b in zip(P, mom)) < 5e-6, (r, P)
        assert abs(j) < 2e-6
        assert abs(m - (1.0 + 1.0 / (2.0 * r))) < 1e-5


def test_trace_term_of_momentum():
    p = idt.centred_patch(48, 0.25)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    k0, k1 = 0.3, 0.05
    u = idt.minkowski(p)
    u[7] = k0 + k1 * x  # Khat; Theta = 0
    for r in (2.0, 4.0):
        m, j, px, py, pz = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), r, 24, 48)
        assert abs(px - (-k1 * r ** 3 / 9.0)) < 1e-12 * r ** 3
        assert abs(py) < 1e-14 and abs(pz) < 1e-14 and abs(j) < 1e-14 and m == 0.0
    # Theta enters K twice: the same trace from Theta = Khat / 2
    u[8] = 0.5 * u[7]
    u[7] = 0.0
    px2 = oracle.adm_integrals(p, u, (0.0, 0.0, 0.0), 2.0, 24, 48)[2]
    assert abs(px2 - (-k1 * 8.0 / 9.0)) < 1e-12 * 8.0


def _gauge_flat(p, eps, x0=(0.3, -0.2, 0.1), sig=2.0):
    """Flat metric plus eps (d_i xi_j + d_j xi_i), xi_i = exp(-|x-x0|^2/sig^2)
    (y, z^2, x y)_i, split into W = det^(-1/6) and gt = W^2 gamma."""
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    X = [x - x0[0], y - x0[1], z - x0[2]]
    e = np.exp(-(X[0] ** 2 + X[1] ** 2 + X[2] ** 2) / sig ** 2)
    P = [y, z * z, x * y]
    zero = 0.0 * x
    dP = [[zero, 1.0 + zero, zero], [zero, zero, 2.0 * z], [y, x, zero]]  # dP[i][j] = d_j p_i
    dxi = [[e * (dP[i][j] - 2.0 * X[j] / sig ** 2 * P[i]) for j in range(3)] for i in range(3)]
    g = np.zeros((3, 3) + x.shape)
    for i in range(3):
        for j in range(3):
            g[i, j] = (1.0 if i == j else 0.0) + eps * (dxi[i][j] + dxi[j][i])
    W = np.linalg.det(np.moveaxis(g, (0, 1), (-2, -1))) ** (-1.0 / 6.0)
    u = idt.minkowski(p)
    u[0] = W
    for a, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        u[1 + a] = W * W * g[i, j]
    return u


def test_pure_gauge_mass_is_second_order():
    p = idt.centred_patch(48, 0.25)
    for r in (2.5, 3.5):
        m1 = oracle.adm_integrals(p, _gauge_flat(p, 1e-3), (0.0, 0.0, 0.0), r, 48, 96)[0]
        m2 = oracle.adm_integrals(p, _gauge_flat(p, 2e-3), (0.0, 0.0, 0.0), r, 48, 96)[0]
        assert abs(m1) < 1e-6
        assert abs(m2 / m1 - 4.0) < 0.4, (r, m1, m2)


def test_sphere_outside_patch_rejected():
    p = idt.centred_patch(32, 0.5)
    with pytest.raises(ValueError):
        oracle.adm_integrals(p, idt.minkowski(p), (0.0, 0.0, 0.0), 8.6, 8, 16)
