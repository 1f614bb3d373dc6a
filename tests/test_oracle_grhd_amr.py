"""Pins of the oracle of the fluid on the Berger-Oliger hierarchy
(oracle/grhd_amr.py; Sec. 2.2.1): the conservative WENO5 prolongation of
the rest-mass density, the restriction by volume average, the reflux.

* WENO5: the two children of a parent cell average to it exactly; on
  smooth data the half-cell averages converge at 5th order (the linear
  weights combine the three quadratic stencils into the 5-cell quartic);
  linear data are reproduced by any weights.
* The fluid's ghost values: a uniform fluid is prolonged exactly; the
  primitives rebuilt from D^ with the child's metric are the parent's.
* Restriction: each parent cell under a child becomes the mean of its 8
  children, the rest of the parent is unchanged.
* The coupled hierarchy (spacetime + fluid on a periodic box with a refined
  patch, a density wave crossing the refinement boundary): with reflux the
  total rest mass of the composite grid is conserved to rounding; without
  it, it is not; the wave keeps its translated profile on both levels."""
import math

import numpy as np
import pytest

import initial_data as idd
import oracle
from oracle import grhd, grhd_amr as A


def _half_avgs(coef, n):
    """Cell averages of the polynomial `coef` over unit cells 0..n-1 and its
    averages over their two halves."""
    P = np.polynomial.polynomial
    anti = P.polyint(coef)

    def avg(a, b):
        return (P.polyval(b, anti) - P.polyval(a, anti)) / (b - a)
    cells = np.array([avg(i - 0.5, i + 0.5) for i in range(n)])
    halves = np.array([avg(i - 0.5, i) if k == 0 else avg(i, i + 0.5) for i in range(n) for k in (0, 1)])
    return cells, halves


def test_weno5_children_are_conservative():
    rng = np.random.default_rng(2)
    q = rng.random((14, 3, 2))
    c = A.weno5_children(q, 0)
    I = np.arange(2, 12)
    assert np.abs(0.5 * (c[2 * I] + c[2 * I + 1]) - q[I]).max() <= 1e-15
    assert np.isnan(c[:4]).all() and np.isnan(c[-4:]).all()


def test_weno5_is_fifth_order_on_smooth_data():
    """Half-cell averages of exp(x) from its cell averages: the error falls
    at 5th order (the linear weights (3/16, 5/8, 3/16) combine the three
    quadratic stencils into the quartic; other weights give 3rd order)."""
    def err(h):
        ctr = (np.arange(14) - 7) * h
        cells = (np.exp(ctr + h / 2) - np.exp(ctr - h / 2)) / h
        left = (np.exp(ctr) - np.exp(ctr - h / 2)) / (h / 2)
        right = (np.exp(ctr + h / 2) - np.exp(ctr)) / (h / 2)
        c = A.weno5_children(cells, 0)
        I = np.arange(2, 12)
        return max(np.abs(c[2 * I] - left[I]).max(), np.abs(c[2 * I + 1] - right[I]).max())
    e = [err(h) for h in (0.1, 0.05, 0.025)]
    assert math.log2(e[0] / e[1]) > 4.8 and math.log2(e[1] / e[2]) > 4.8, e
    # linear data: every stencil is exact, whatever the weights
    cells, halves = _half_avgs([2.0, 0.3], 14)
    c = A.weno5_children(cells, 0)
    I = np.arange(2, 12)
    idx = np.concatenate([2 * I, 2 * I + 1])
    assert np.abs(c[idx] - halves[idx]).max() <= 1e-14


def _two_level(n0=24, nc=16, off=8):
    dx0 = 1.0 / n0
    P0 = idd.Patch(n=(n0, n0, n0), dx=dx0, origin=(-0.5, -0.5, -0.5), level=0)
    C1 = idd.Patch(n=(nc, nc, nc), dx=dx0 / 2, origin=tuple(-0.5 + off * dx0 for _ in range(3)), level=1)
    return idd.Hierarchy(dx0=dx0, levels=[[P0], [C1]], masses=[], positions=[]), P0, C1


GAS = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)


def test_uniform_fluid_prolongs_exactly():
    h, P0, C1 = _two_level()
    cons = np.zeros((5,) + P0.shape[1:])
    prim = np.zeros((5,) + P0.shape[1:])
    cons[0], prim[1], prim[2], prim[3], prim[4] = 2e-6, 0.4, 0.1, -0.2, 0.05
    v = A.prolong_fluid(P0, cons, prim, C1)
    m = A.ghost_mask(C1)
    for f, want in enumerate([2e-6, 0.4, 0.1, -0.2, 0.05]):
        assert np.abs(v[f][m] - want).max() <= 1e-15 * max(abs(want), 1e-6)
    assert np.isnan(v[:, ~m]).all()
    # the primitives from D^ with a (flat) child metric
    u = idd.minkowski(C1)
    gp = A.ghost_primitives(v, C1, u, GAS)
    w = math.sqrt(1.0 + 0.1 ** 2 + 0.2 ** 2 + 0.05 ** 2)
    assert np.abs(gp[0][m] - 2e-6 / w).max() <= 1e-15 * 2e-6


def test_restriction_is_the_volume_average():
    h, P0, C1 = _two_level()
    rng = np.random.default_rng(4)
    cp = rng.random((5,) + P0.shape[1:])
    cc = rng.random((5,) + C1.shape[1:])
    out = A.restrict_fluid(P0, cp, C1, cc)
    g, off = P0.g, A.child_offset(P0, C1)
    for (K, J, I) in [(0, 0, 0), (3, 5, 7), (7, 7, 7)]:
        ch = cc[:, g + 2 * K:g + 2 * K + 2, g + 2 * J:g + 2 * J + 2, g + 2 * I:g + 2 * I + 2]
        assert np.allclose(out[:, g + off[2] + K, g + off[1] + J, g + off[0] + I], ch.mean(axis=(1, 2, 3)),
                           rtol=1e-15, atol=0)
    mask = np.ones(P0.shape[1:], dtype=bool)
    mask[g + off[2]:g + off[2] + 8, g + off[1]:g + off[1] + 8, g + off[0]:g + off[0] + 8] = False
    assert np.array_equal(out[:, mask], cp[:, mask])


def _wave_hierarchy(reflux):
    h, P0, C1 = _two_level()
    v, W = 0.3, 1.0 / math.sqrt(1.0 - 0.09)

    def fluid(p, t=0.0):
        x = p.axis(0)
        pr = np.zeros((5,) + p.shape[1:])
        pr[0] = (1e-6 * (1.0 + 0.2 * np.sin(2.0 * np.pi * (x - v * t))))[None, None, :]
        pr[1] = 1e-7 / ((5.0 / 3.0 - 1.0) * pr[0])
        pr[2] = W * v
        return pr
    H = A.MatterHierarchy(h, [idd.minkowski(p) for p in (P0, C1)], [fluid(p) for p in (P0, C1)], GAS,
                          [np.full(p.shape[1:], 1e-18) for p in (P0, C1)], oracle.Params(lapse=1, shift=1),
                          courant=0.25, bc0=oracle.BC_PERIODIC, reflux=reflux)
    return H, (P0, C1), fluid


@pytest.fixture(scope="module")
def wave_runs():
    out = {}
    for refl in (True, False):
        H, ps, fluid = _wave_hierarchy(refl)
        m0 = H.rest_mass()
        for _ in range(3):
            H.level_step(0)
        out[refl] = (H, ps, fluid, m0)
    return out


def test_reflux_conserves_the_rest_mass(wave_runs):
    H, _, _, m0 = wave_runs[True]
    assert abs(H.rest_mass() - m0) <= 2e-15 * m0
    H, _, _, m0 = wave_runs[False]
    assert abs(H.rest_mass() - m0) > 1e-9 * m0


def test_wave_crosses_the_refinement_boundary(wave_runs):
    """After three coarse steps (t = 0.094, the wave moved 1.4 parent cells)
    the density on both levels is the translated profile to 2% of the
    wave's amplitude (2e-7)."""
    H, ps, fluid, _ = wave_runs[True]
    t = 3 * H.dt(0)
    for pid, p in enumerate(ps):
        g = p.g
        got = H.prim(pid)[0, g:-g, g:-g, g:-g]
        want = fluid(p, t)[0, g:-g, g:-g, g:-g]
        assert np.abs(got - want).max() <= 0.02 * 2e-7, (pid, np.abs(got - want).max())
