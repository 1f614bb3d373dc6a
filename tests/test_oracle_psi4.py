"""Pins of the oracle's Psi4 extraction (Sec. 2.3) against closed forms.

* _{-2}Y_lm: the closed forms of l = 2 (e.g. sqrt(5/(64 pi)) (1 + cos th)^2
  e^{2 i phi} for m = 2) and orthonormality up to l = 6 under an exact
  quadrature.
* A linearised plane wave h_+ = A sin(w u), h_x = B cos(w u), u = t - k.x,
  along several directions k: at the sphere point in direction k,
  Psi4 = -d_t^2 (h_+ - i h_x) (the convention of h = -int int Psi4), to 4th
  order in dx (the triad errors are second order in the amplitude).  A wrong
  sign of B_ij, a transposed epsilon or a missing K K term would show as an
  O(1) relative error.
* Schwarzschild (one Brill-Lindquist puncture): Psi4 = 0 in the radial
  triad (type D), reached at 4th order.
* The l = 2 modes of the plane wave along z against an independent numpy
  quadrature of its closed-form Psi4 on the sphere (linearised E and B in
  the flat triad) with the closed-form harmonics.
"""
import math

import numpy as np
import pytest

import initial_data as idd
import oracle


def _y2(m, th, ph):
    c = math.cos(th)
    s = math.sin(th)
    amp = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2, 1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
           0: math.sqrt(15 / (32 * math.pi)) * s * s, -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
           -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}[m]
    return amp * complex(math.cos(m * ph), math.sin(m * ph))


def test_swsh_closed_forms_l2():
    rng = np.random.default_rng(4)
    for _ in range(10):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        for m in range(-2, 3):
            assert abs(oracle.swsh(2, m, th, ph) - _y2(m, th, ph)) < 1e-14


def test_swsh_orthonormal():
    x, w = np.polynomial.legendre.leggauss(40)
    nph = 80
    phis = 2 * math.pi * np.arange(nph) / nph
    lm = [(l, m) for l in range(2, 7) for m in range(-l, l + 1)]
    Y = np.array([[[oracle.swsh(l, m, math.acos(c), ph) for ph in phis] for c in x] for (l, m) in lm])
    G = np.einsum("ath,bth,t->ab", Y, Y.conj(), w) * (2 * math.pi / nph)
    assert np.abs(G - np.eye(len(lm))).max() < 1e-12


def _plane_psi4(A, B, w, k, x):
    uu = -np.dot(k, x)
    return complex(A * w * w * math.sin(w * uu), -B * w * w * math.cos(w * uu))  # -(h+'' - i hx'')


@pytest.mark.parametrize("direction", [(0.7, 0.3), (2.0, -1.2), (1.2, 2.5)])
def test_plane_wave_pointwise_fourth_order(direction):
    A, B, w, r = 1e-6, 0.6e-6, 1.0, 1.5
    th, ph = direction
    k, _, _ = idd.plane_wave_basis(th, ph)
    exp = _plane_psi4(A, B, w, k, r * k)
    errs = []
    for n in (32, 64):
        p = idd.centred_patch(n, 8.0 / n)
        u = idd.plane_wave(p, A, B, w, th, ph)
        errs.append(abs(oracle.psi4_point(p, u, (0.0, 0.0, 0.0), r, th, ph) - exp) / abs(exp))
    assert errs[1] < 1e-5 and errs[0] / errs[1] > 6, errs  # 4th order: 16; 2nd order would be 4


def test_schwarzschild_psi4_vanishes():
    vals = []
    for n in (32, 64):
        p = idd.centred_patch(n, 16.0 / n)
        u = idd.bowen_york(p, 1.0)
        m = oracle.psi4_modes(p, u, (0.0, 0.0, 0.0), 5.0, 16, 32, 4)
        vals.append(max(abs(v) for v in m.values()))
    # E_ij itself is of order M / r^3 = 8e-3 here
    assert vals[1] < 1e-6 and vals[0] / vals[1] > 10, vals


def test_plane_wave_modes_against_closed_form():
    A, B, w, r = 1e-6, 0.4e-6, 1.2, 2.0
    p = idd.centred_patch(64, 0.125)
    u = idd.plane_wave(p, A, B, w, 0.0, 0.0)  # along z, e1 = x, e2 = y
    k = np.array([0.0, 0.0, 1.0])
    modes = oracle.psi4_modes(p, u, (0.0, 0.0, 0.0), r, 24, 48, 2)
    # linearised E, B of the wave at x, contracted with the flat triad
    x, wg = np.polynomial.legendre.leggauss(60)
    nph = 120
    ref = {m: 0j for m in range(-2, 3)}
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    e1, e2 = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    Ep, Ex = np.outer(e1, e1) - np.outer(e2, e2), np.outer(e1, e2) + np.outer(e2, e1)
    for c, wt in zip(x, wg):
        th = math.acos(c)
        for j in range(nph):
            ph = 2 * math.pi * j / nph
            n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), c])
            uu = -np.dot(k, r * n)
            hdd = -A * w * w * math.sin(w * uu) * Ep - B * w * w * math.cos(w * uu) * Ex
            E = -0.5 * hdd
            C = 0.5 * np.einsum("ikl,k,lj->ij", eps, k, hdd)
            Bm = 0.5 * (C + C.T)
            et = np.array([c * math.cos(ph), c * math.sin(ph), -math.sin(th)])
            ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
            mb = (et - 1j * ep) / math.sqrt(2)
            psi = mb @ (E - 1j * Bm) @ mb
            for m in range(-2, 3):
                ref[m] += wt * (2 * math.pi / nph) * psi * _y2(m, th, ph).conjugate()
    scale = max(abs(v) for v in ref.values())
    assert scale > 1e-7
    for m in range(-2, 3):
        assert abs(modes[(2, m)] - ref[m]) < 1e-4 * scale, (m, modes[(2, m)], ref[m])


def test_psi4_rejects_sphere_outside():
    p = idd.centred_patch(32, 0.5)
    with pytest.raises(ValueError):
        oracle.psi4_modes(p, idd.minkowski(p), (0.0, 0.0, 0.0), 8.6, 8, 16, 2)
    assert all(v == 0 for v in oracle.psi4_modes(p, idd.minkowski(p), (0.0, 0.0, 0.0), 5.0, 8, 16, 3).values())
