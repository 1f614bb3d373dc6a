"""Pins of the oracle's Berger-Oliger operators (Sec. 2.2.1): 6th-order
Lagrange prolongation (exact on degree <= 5), 4th-order restriction (exact on
degree <= 3), the interpolation weights as exact fractions, the time
interpolant (exact on quadratics), the same-level exchange rules, and the
subcycling driver on the gauge wave."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import initial_data as idd
import oracle


def _lagrange_fraction(nodes, x):
    w = []
    for j, tj in enumerate(nodes):
        v = Fraction(1)
        for m, tm in enumerate(nodes):
            if m != j:
                v *= (x - tm) / Fraction(tj - tm)
        w.append(v)
    return w


def test_prolongation_weights_exact_fractions():
    w = oracle.lagrange_weights([-2, -1, 0, 1, 2, 3], 0.25)
    assert list(w * 8192) == [77, -693, 6930, 2310, -495, 63]
    w = oracle.lagrange_weights([-3, -2, -1, 0, 1, 2], -0.25)
    assert list(w * 8192) == [63, -495, 2310, 6930, -693, 77]
    w = oracle.lagrange_weights([-1, 0, 1, 2], 0.5)
    assert list(w * 16) == [-1, 9, 9, -1]
    for nodes, x in [([-1, 0, 1], Fraction(1, 4)), ([-1, 0, 1], Fraction(3, 4))]:
        exact = [float(v) for v in _lagrange_fraction(nodes, x)]
        assert list(oracle.lagrange_weights(nodes, float(x))) == exact


def _parent_child():
    parent = idd.Patch(n=(16, 16, 16), dx=0.5, origin=(-4.0, -4.0, -4.0))
    child = idd.Patch(n=(8, 10, 12), dx=0.25, origin=(-1.0, -1.5, -1.0), level=1)
    return parent, child


def _fill(p, fn):
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    u = np.zeros(p.shape)
    for f in range(25):
        u[f] = fn(x, y, z) * (1 + f)
    return u


@pytest.mark.parametrize("a,b,c", [(5, 0, 0), (0, 5, 0), (0, 0, 5), (2, 3, 1), (5, 5, 5), (1, 4, 2), (0, 0, 0)])
def test_prolongation_exact_on_degree_5(a, b, c):
    parent, child = _parent_child()
    fn = lambda x, y, z: (x + 0.3) ** a * (y - 0.2) ** b * (z + 0.1) ** c
    up = _fill(parent, fn)
    uc = oracle.prolong_ghosts(parent, up, child, np.zeros(child.shape))
    ex = _fill(child, fn)
    g = child.g
    ghost = np.ones(child.shape[1:], bool)
    ghost[g:-g, g:-g, g:-g] = False
    scale = np.abs(ex).max()
    np.testing.assert_allclose(uc[:, ghost], ex[:, ghost], rtol=0, atol=1e-11 * scale)
    assert np.all(uc[:, ~ghost] == 0.0)  # active points untouched


def test_prolongation_not_exact_on_degree_6():
    parent, child = _parent_child()
    fn = lambda x, y, z: (x + 0.3) ** 6
    uc = oracle.prolong_ghosts(parent, _fill(parent, fn), child, np.zeros(child.shape))
    ex = _fill(child, fn)
    assert np.abs(uc[:, :3] - ex[:, :3]).max() > 1e-6


@pytest.mark.parametrize("a,b,c", [(3, 0, 0), (0, 3, 0), (0, 0, 3), (1, 2, 3), (3, 3, 3), (0, 0, 0)])
def test_restriction_exact_on_degree_3(a, b, c):
    parent, child = _parent_child()
    fn = lambda x, y, z: (x - 0.4) ** a * (y + 0.7) ** b * (z - 0.15) ** c
    uc = _fill(child, fn)
    up0 = np.full(parent.shape, -7.0)
    up = oracle.restrict(parent, up0, child, uc)
    ex = _fill(parent, fn)
    changed = up != -7.0
    # exactly the parent cells covered by the child's active region
    assert changed[0].sum() == (8 // 2) * (10 // 2) * (12 // 2)
    np.testing.assert_allclose(up[changed], ex[changed], rtol=1e-12, atol=1e-12)


def test_restriction_not_exact_on_degree_4():
    parent, child = _parent_child()
    fn = lambda x, y, z: (x - 0.4) ** 4
    up = oracle.restrict(parent, np.full(parent.shape, -7.0), child, _fill(child, fn))
    ex = _fill(parent, fn)
    changed = up != -7.0
    assert np.abs(up[changed] - ex[changed]).max() > 1e-6


def test_misaligned_child_rejected():
    parent, child = _parent_child()
    bad = idd.Patch(n=child.n, dx=child.dx, origin=(-1.0 + child.dx, -1.5, -1.0))
    with pytest.raises(ValueError):
        oracle.prolong_ghosts(parent, np.zeros(parent.shape), bad, np.zeros(bad.shape))


def test_time_interpolation_exact_on_quadratics():
    """Parent levels at t-DT, t, t+DT (oldest first); fraction s of the last
    step: quadratic weights reproduce any quadratic in time; linear weights
    (two levels) reproduce linear functions (Sec. 2.2.1)."""
    q = lambda t: 0.3 - 1.7 * t + 2.2 * t * t
    for s in (0.0, 0.25, 0.5, 0.75, 1.0):
        w = oracle.time_weights(3, s)
        assert w @ np.array([q(-1.0), q(0.0), q(1.0)]) == pytest.approx(q(s), rel=1e-15, abs=1e-15)
        w = oracle.time_weights(2, s)
        lin = lambda t: 0.4 + 3.0 * t
        assert w @ np.array([0.0, lin(0.0), lin(1.0)]) == pytest.approx(lin(s), rel=1e-15)
    assert list(oracle.time_weights(3, 0.25)) == [-3 / 32, 15 / 16, 5 / 32]


def test_exchange_rules_brute_force():
    """Ghosts over the other patch's active region are overwritten by it;
    active points present in both patches become the average; the rest is
    untouched (Sec. 2.2.1)."""
    a = idd.Patch(n=(6, 4, 4), dx=0.5, origin=(0.0, 0.0, 0.0))
    b = idd.Patch(n=(6, 4, 4), dx=0.5, origin=(2.0, 0.0, 0.0))  # overlaps a's cells 4,5
    rng = np.random.default_rng(5)
    ua0 = rng.standard_normal(a.shape)
    ub0 = rng.standard_normal(b.shape)
    ua, ub = ua0.copy(), ub0.copy()
    n = oracle.exchange(a, ua, b, ub)
    assert n > 0
    g = 3
    for ia in range(-g, 6 + g):
        ib = ia - 4
        for j in range(-g, 4 + g):
            for k in range(-g, 4 + g):
                qa = (slice(None), k + g, j + g, ia + g)
                a_act = 0 <= ia < 6 and 0 <= j < 4 and 0 <= k < 4
                b_in = -g <= ib < 6 + g
                b_act = 0 <= ib < 6 and 0 <= j < 4 and 0 <= k < 4
                if not b_in:
                    assert np.array_equal(ua[qa], ua0[qa])
                    continue
                qb = (slice(None), k + g, j + g, ib + g)
                if a_act and b_act:
                    np.testing.assert_array_equal(ua[qa], 0.5 * (ua0[qa] + ub0[qb]))
                    np.testing.assert_array_equal(ub[qb], ua[qa])
                elif b_act:
                    np.testing.assert_array_equal(ua[qa], ub0[qb])
                elif a_act:
                    np.testing.assert_array_equal(ub[qb], ua0[qa])
                else:
                    assert np.array_equal(ua[qa], ua0[qa]) and np.array_equal(ub[qb], ub0[qb])


# ------------------------------------------------------------------ driver

def _gw_hierarchy(n0):
    """Periodic unit box with two nested levels, each half the parent's width."""
    levels = [[idd.Patch(n=(n0, n0, n0), dx=1.0 / n0, origin=(-0.5, -0.5, -0.5), level=0)]]
    for l in (1, 2):
        dx = 1.0 / n0 / 2 ** l
        levels.append([idd.centred_patch(n0, dx, level=l)])
    return idd.Hierarchy(dx0=1.0 / n0, levels=levels, masses=[], positions=[])


def _gw_amr_errors(n0, coarse_steps, amp=0.01, history=True):
    h = _gw_hierarchy(n0)
    prm = oracle.Params(lapse=1, shift=1, sigma_ko=0.0, kappa1=0.0)
    states = [idd.gauge_wave(p, amp) for p in h.patches]
    prev = None
    if history:
        prev = []
        for p in h.patches:
            u = idd.gauge_wave(p, amp, t=-0.25 * h.dx0 / 2 ** p.level)
            prev.append(oracle.fill_periodic(p, u) if p.level == 0 else u)
    bo = oracle.BOHierarchy(h, states, prm, courant=0.25, bc0=oracle.BC_PERIODIC, previous=prev)
    for _ in range(coarse_steps):
        bo.level_step(0)
    T = coarse_steps * 0.25 / n0
    errs = []
    for pid, p in enumerate(h.patches):
        ex = idd.gauge_wave(p, amp, t=T)
        g = p.g
        errs.append(np.abs(bo.current(pid)[:, g:-g, g:-g, g:-g] - ex[:, g:-g, g:-g, g:-g]).max())
    return errs, T


def test_bo_driver_gauge_wave():
    """Three nested levels of the gauge wave in a periodic box.  With the
    previous time level supplied (so every ghost fill uses the quadratic time
    interpolant) the hierarchy converges at 2nd order at fixed physical time:
    refilling refinement-boundary ghosts at every RK stage with interpolated
    parent data is 2nd-order consistent at the interface.  A wrong stage time,
    time weight or parent pairing leaves O(A dt) errors that do not converge.
    Without history the very first step interpolates linearly (Sec. 2.2.1) and
    the error stays bounded at the 1e-4 level."""
    e16, _ = _gw_amr_errors(16, 2)
    e32, _ = _gw_amr_errors(32, 4)
    assert max(e16) < 2e-5, e16
    assert math.log2(max(e16) / max(e32)) > 1.5, (e16, e32)
    e_lin, _ = _gw_amr_errors(16, 2, history=False)
    assert max(e_lin) < 5e-4, e_lin


# ------------------------------------------------------------------ two patches on a level

def _split_merged(split):
    """3 levels: L0 32^3 (dx 1), L1 one 32x16x16 patch on [-8,8]x[-4,4]^2 or the
    same region as two abutting 16^3 patches (split at x = 0), L2 8^3 (dx 1/4)
    inside the right half."""
    l0 = [idd.Patch(n=(32, 32, 32), dx=1.0, origin=(-16.0, -16.0, -16.0), level=0)]
    if split:
        l1 = [idd.Patch(n=(16, 16, 16), dx=0.5, origin=(-8.0, -4.0, -4.0), level=1),
              idd.Patch(n=(16, 16, 16), dx=0.5, origin=(0.0, -4.0, -4.0), level=1)]
    else:
        l1 = [idd.Patch(n=(32, 16, 16), dx=0.5, origin=(-8.0, -4.0, -4.0), level=1)]
    l2 = [idd.Patch(n=(8, 8, 8), dx=0.25, origin=(3.0, -1.0, -1.0), level=2)]
    h = idd.Hierarchy(dx0=1.0, levels=[l0, l1, l2], masses=[0.3], positions=[(4.05, 0.1, -0.15)])
    return h, idd.hierarchy_data(h, noise=1e-6, seed=7)


def test_bo_split_level_equals_merged_level():
    """A level made of two abutting patches evolves exactly like the single
    patch covering the same cells (Sec. 2.2.1): at every stage each patch's
    ghosts over the neighbour's active cells take the neighbour's values
    (exchange after the prolongation), and after the two child steps the
    ghosts are refilled at the parent's new time, exchanged and only then
    restricted.  Any other order leaves prolonged values where the merged
    patch has evolved ones, and the two runs part at O(1e-6) (the noise)."""
    hs, us = _split_merged(True)
    hm, um = _split_merged(False)
    prm = oracle.Params()
    bs = oracle.BOHierarchy(hs, us, prm, courant=0.25)
    bm = oracle.BOHierarchy(hm, um, prm, courant=0.25)
    for _ in range(2):
        bs.level_step(0)
        bm.level_step(0)
    g = 3
    act = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    scale = np.abs(bm.current(0)[act]).max()
    for a, b in ((0, 0), (3, 2)):  # L0 and L2 patches
        d = np.abs(bs.current(a)[act] - bm.current(b)[act]).max()
        assert d <= 1e-14 * scale, (a, d)
    merged = bm.current(1)
    for pid, x0 in ((1, 0), (2, 16)):  # the halves inside the merged patch
        part = merged[:, g:-g, g:-g, g + x0:g + x0 + 16]
        d = np.abs(bs.current(pid)[act] - part).max()
        assert d <= 1e-14 * scale, (pid, d)
    # the runs did evolve the noise (the pin is not vacuous)
    assert np.abs(bm.current(1)[act] - um[1][act]).max() > 1e-4
