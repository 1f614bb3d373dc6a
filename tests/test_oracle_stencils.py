"""Pins of the oracle's finite-difference operators (Sec. 2.2): exactness on
polynomials up to each stencil's order, the upwind bias following the sign of
the shift, and the Kreiss-Oliger operator's closed form on x^6."""
import itertools

import numpy as np
import pytest

import initial_data as idd
import oracle


def _poly_patch():
    return idd.Patch(n=(8, 8, 8), dx=0.25, origin=(-1.0, -0.75, -0.5))


def _field_from(p, fn):
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    u = np.zeros(p.shape)
    u[7] = fn(x, y, z)
    return u, (x, y, z)


@pytest.mark.parametrize("a,b,c", [(1, 0, 0), (2, 1, 0), (4, 0, 0), (0, 4, 0), (0, 0, 4), (3, 1, 0),
                                   (2, 2, 0), (0, 3, 1), (1, 1, 2)])
def test_first_derivatives_exact_to_degree_4(a, b, c):
    p = _poly_patch()
    u, (x, y, z) = _field_from(p, lambda x, y, z: x ** a * y ** b * z ** c)
    for (i, j, k) in [(4, 5, 6), (6, 3, 5), (5, 5, 5)]:
        s = oracle.stencils(p, u, 7, i, j, k)
        X, Y, Z = x[k, j, i], y[k, j, i], z[k, j, i]
        ex = [a * X ** max(a - 1, 0) * Y ** b * Z ** c,
              b * X ** a * Y ** max(b - 1, 0) * Z ** c,
              c * X ** a * Y ** b * Z ** max(c - 1, 0)]
        np.testing.assert_allclose(s[0:3], ex, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_second_derivatives_exact_to_degree_5(deg):
    p = _poly_patch()
    u, (x, y, z) = _field_from(p, lambda x, y, z: x ** deg + 2 * y ** deg - z ** deg)
    i, j, k = 5, 6, 4
    s = oracle.stencils(p, u, 7, i, j, k)
    X, Y, Z = x[k, j, i], y[k, j, i], z[k, j, i]
    d2 = lambda t: deg * (deg - 1) * t ** max(deg - 2, 0)
    np.testing.assert_allclose(s[3:6], [d2(X), 2 * d2(Y), -d2(Z)], rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("a,b", list(itertools.product(range(5), range(5))))
def test_nested_mixed_derivative_exact(a, b):
    p = _poly_patch()
    u, (x, y, z) = _field_from(p, lambda x, y, z: x ** a * y ** b + y ** a * z ** b + x ** b * z ** a)
    i, j, k = 5, 4, 6
    s = oracle.stencils(p, u, 7, i, j, k)
    X, Y, Z = x[k, j, i], y[k, j, i], z[k, j, i]
    dp = lambda t, e: e * t ** max(e - 1, 0)
    exy = dp(X, a) * dp(Y, b)
    exz = dp(X, b) * dp(Z, a)
    eyz = dp(Y, a) * dp(Z, b)
    np.testing.assert_allclose(s[6:9], [exy, exz, eyz], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_upwind_exact_to_degree_4(sign, deg):
    p = _poly_patch()
    u, (x, y, z) = _field_from(p, lambda x, y, z: (x - 0.1) ** deg + (y + 0.2) ** deg + z ** deg)
    i, j, k = 5, 5, 5
    s = oracle.stencils(p, u, 7, i, j, k, b=(sign, sign, sign))
    X, Y, Z = x[k, j, i], y[k, j, i], z[k, j, i]
    ex = [deg * (X - 0.1) ** (deg - 1), deg * (Y + 0.2) ** (deg - 1), deg * Z ** (deg - 1)]
    np.testing.assert_allclose(s[9:12], ex, rtol=1e-11, atol=1e-11)


def test_upwind_bias_follows_shift_sign():
    """On f = (x - x0)^6 at x = x0 the lopsided stencil one-behind/three-ahead
    gives (-3 + 18 - 6*64 + 729)/12 h^5 = +30 h^5; the mirrored one gives -30 h^5."""
    p = _poly_patch()
    i, j, k = 5, 5, 5
    x0 = p.axis(0)[i]
    u, _ = _field_from(p, lambda x, y, z: (x - x0) ** 6)
    h = p.dx
    s_pos = oracle.stencils(p, u, 7, i, j, k, b=(0.7, 0.0, 0.0))
    s_neg = oracle.stencils(p, u, 7, i, j, k, b=(-0.7, 0.0, 0.0))
    assert s_pos[9] == pytest.approx(30 * h ** 5, rel=1e-12)
    assert s_neg[9] == pytest.approx(-30 * h ** 5, rel=1e-12)


def test_sixth_difference_closed_form():
    """Delta^6 annihilates degree <= 5 and gives 6! h^6 on x^6."""
    p = _poly_patch()
    h = p.dx
    u, _ = _field_from(p, lambda x, y, z: x ** 5 - 3 * y ** 4 + z ** 3 + x * y * z)
    s = oracle.stencils(p, u, 7, 5, 5, 5)
    np.testing.assert_allclose(s[12:15], 0.0, atol=1e-11)
    u, _ = _field_from(p, lambda x, y, z: x ** 6 + 2 * y ** 6 - z ** 6)
    s = oracle.stencils(p, u, 7, 5, 5, 5)
    np.testing.assert_allclose(s[12:15], np.array([1, 2, -1]) * 720 * h ** 6, rtol=1e-9)


def test_ko_term_in_rhs():
    """The dissipation added to a field's RHS is sigma/(64 h) sum_dirs Delta^6 f
    (Sec. 2.2, sigma = 0.5): on f = x^6 + y^6 + z^6 it is 3 sigma 720 h^5 / 64."""
    p = _poly_patch()
    u = idd.minkowski(p)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    u[8] = x ** 6 + y ** 6 + z ** 6
    prm = oracle.Params(sigma_ko=0.5)
    r = oracle.rhs(p, u, prm, terms=4)
    h = p.dx
    g = p.g
    act = r[8, g:-g, g:-g, g:-g]
    np.testing.assert_allclose(act, 3 * 0.5 * 720 * h ** 5 / 64.0, rtol=1e-8)
    # dissipation never leaks into other fields
    assert np.abs(np.delete(r, 8, axis=0)).max() == 0.0


def test_advection_term_in_rhs():
    """The advection term is beta^j d_j f for every field (Sec. 2.2): exact for a
    quadratic f and constant shift of either sign."""
    p = _poly_patch()
    u = idd.minkowski(p)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    bet = (0.3, -0.2, 0.1)
    for d in range(3):
        u[19 + d] = bet[d]
    u[9] = x * x - 2 * x * y + 3 * z
    r = oracle.rhs(p, u, oracle.Params(), terms=2)
    g = p.g
    ex = bet[0] * (2 * x - 2 * y) + bet[1] * (-2 * x) + bet[2] * 3.0
    np.testing.assert_allclose(r[9, g:-g, g:-g, g:-g], ex[g:-g, g:-g, g:-g], rtol=1e-12, atol=1e-13)
