"""Pin of every term of the oracle's Z4c RHS and constraint monitor: on smooth
generic data (non-flat conformal metric, non-zero K_ij, lapse, shift and B)
the discrete values must converge at 4th order (Sec. 2.2) to the continuum
values computed from the ADM equations by an independent route
(tests/continuum.py: physical Christoffels and Ricci by definition, exact
derivatives by autograd).  A dropped term, a wrong sign or a transposed index
leaves an O(1) residual that does not converge."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import initial_data as idd
import oracle

from tests import continuum as C


def _grid_points(p):
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _state(p):
    pts = _grid_points(p)
    vals = C.on_points(C.z4c_state, pts)  # (N, 25)
    return np.ascontiguousarray(vals.T.reshape(p.shape))


def _sample(p):
    """About 8^3 active points spread over the patch (every (n/8)-th cell)."""
    g = p.g
    st = max(p.n[0] // 8, 1)
    return slice(g, g + p.n[0], st)


def _active(p, a):
    s = _sample(p)
    return a[..., s, s, s]


def _active_points(p):
    s = _sample(p)
    z, y, x = np.meshgrid(p.axis(2)[s], p.axis(1)[s], p.axis(0)[s], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


@pytest.fixture(scope="module")
def runs():
    out = {}
    for n in (16, 32):
        p = idd.Patch(n=(n, n, n), dx=1.0 / n, origin=(-0.5, -0.5, -0.5))
        u = _state(p)
        prm = oracle.Params(sigma_ko=0.0, kappa1=0.005, eta=0.36)
        r = _active(p, oracle.rhs(p, u, prm)).reshape(25, -1)
        ex = C.on_points(lambda x: C.z4c_rhs_continuum(x, eta=0.36), _active_points(p)).T
        c, _ = oracle.constraints(p, u)
        cc = _active(p, c).reshape(4, -1)
        cex = C.on_points(C.constraints_continuum, _active_points(p)).T
        out[n] = (r, ex, cc, cex)
    return out


def test_data_is_generic(runs):
    """Every field's continuum RHS is O(0.01-1), so no term is trivially zero."""
    r, ex, _, cex = runs[16]
    mags = np.abs(ex).max(axis=1)
    assert (mags > 1e-3).all(), mags
    assert (np.abs(cex).max(axis=1) > 1e-3).all()


@pytest.mark.parametrize("f", range(25), ids=idd.FIELD_NAMES)
def test_rhs_converges_4th_order(runs, f):
    e = []
    for n in (16, 32):
        r, ex, _, _ = runs[n]
        e.append(np.abs(r[f] - ex[f]).max())
    scale = np.abs(runs[32][1][f]).max()
    rate = np.log2(e[0] / e[1])
    assert e[1] < 2e-3 * scale, (e, scale)
    assert rate > 3.5, (e, rate)


@pytest.mark.parametrize("c", range(4), ids=["H", "Mx", "My", "Mz"])
def test_constraints_converge_4th_order(runs, c):
    e = []
    for n in (16, 32):
        _, _, cc, cex = runs[n]
        e.append(np.abs(cc[c] - cex[c]).max())
    scale = np.abs(runs[32][3][c]).max()
    rate = np.log2(e[0] / e[1])
    assert e[1] < 2e-3 * scale, (e, scale)
    assert rate > 3.5, (e, rate)
