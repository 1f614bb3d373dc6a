"""Pins of the oracle's moving boxes (Sec. 2.2.1): puncture tracking
dx/dt = -beta(x), patch shifts in steps of two cells with the newly covered
region prolonged from the parent, and the regrid rule.

* orc_interp_point: exact on tricubic polynomials, not on quartics.
* orc_move_patch: cells that were active keep their values bit for bit; the
  others are the parent's 6th-order prolongation, exact on degree-5
  polynomials (brute-force check of every cell); misalignment is rejected.
* Tracking: with a uniform shift b on periodic Minkowski data the puncture
  moves exactly as x0 - b t; with a static linear shift
  beta^x = -a (x - xs) the exact solution is xs + (x0 - xs) exp(a t) and
  Heun's method converges at second order.
* Regrid: afterwards every following patch has its puncture within one
  parent cell of its centre, every patch nests, and the level's time-level
  history restarts.
"""
import math

import numpy as np
import pytest

import initial_data as idd
import oracle


def _poly(p, deg, seed=3):
    """Every field = a random polynomial of total degree deg in x, y, z."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    u = np.zeros(p.shape)
    for f in range(idd.NF):
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                c = deg - a - b
                u[f] += rng.uniform(-1, 1) * (x / 4) ** a * (y / 4) ** b * (z / 4) ** c
        u[f] += 2.0
    return u


def test_interp_point_exact_on_tricubics():
    p = idd.Patch(n=(12, 10, 14), dx=0.5, origin=(-3.0, -2.5, -3.5))
    rng = np.random.default_rng(0)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    cf = rng.uniform(-1, 1, (4, 4, 4))
    u = np.zeros(p.shape)
    u[20] = sum(cf[a, b, c] * x ** a * y ** b * z ** c for a in range(4) for b in range(4) for c in range(4))
    u[7] = x ** 4
    for _ in range(20):
        q = rng.uniform([-2.2, -1.7, -2.7], [2.2, 1.7, 2.7])
        exact = sum(cf[a, b, c] * q[0] ** a * q[1] ** b * q[2] ** c
                    for a in range(4) for b in range(4) for c in range(4))
        assert abs(oracle.interp_point(p, u, 20, q) - exact) < 1e-11 * (1 + abs(exact))
    # a quartic is not reproduced away from the nodes
    assert abs(oracle.interp_point(p, u, 7, (0.1, 0.0, 0.0)) - 0.1 ** 4) > 1e-6
    with pytest.raises(ValueError):  # the stencil would need a ghost cell
        oracle.interp_point(p, u, 7, (-2.6, 0.0, 0.0))


def _parent_child():
    par = idd.Patch(n=(24, 24, 24), dx=1.0, origin=(-12.0, -12.0, -12.0), level=0)
    old = idd.Patch(n=(16, 12, 14), dx=0.5, origin=(-4.0, -3.0, -3.0), level=1)
    return par, old


@pytest.mark.parametrize("shift", [(1, 0, 0), (-2, 1, 0), (0, -1, 2), (3, 3, -3)])
def test_move_patch_copies_and_prolongs(shift):
    par, old = _parent_child()
    up = _poly(par, 5)
    rng = np.random.default_rng(1)
    uo = rng.uniform(-1, 1, old.shape)  # old data unrelated to the parent
    new = idd.Patch(n=old.n, dx=old.dx, level=1,
                    origin=tuple(old.origin[d] + 2 * shift[d] * old.dx for d in range(3)))
    un = oracle.move_patch(par, up, old, uo, new)
    ref = _poly(new, 5)
    g = new.g
    sh = [2 * s for s in shift]
    n_copy = n_prol = 0
    for k in range(new.shape[1]):
        for j in range(new.shape[2]):
            for i in range(new.shape[3]):
                io, jo, ko = i + sh[0], j + sh[1], k + sh[2]
                if g <= io < g + old.n[0] and g <= jo < g + old.n[1] and g <= ko < g + old.n[2]:
                    assert np.array_equal(un[:, k, j, i], uo[:, ko, jo, io])
                    n_copy += 1
                else:
                    assert np.abs(un[:, k, j, i] - ref[:, k, j, i]).max() < 1e-12
                    n_prol += 1
    assert n_copy > 0 and n_prol > 0
    # degree 6 is not reproduced by the prolongation
    un6 = oracle.move_patch(par, _poly(par, 6), old, uo, new)
    assert np.abs(un6[:, 0] - _poly(new, 6)[:, 0]).max() > 1e-9


def test_move_patch_rejects_misalignment():
    par, old = _parent_child()
    bad = idd.Patch(n=old.n, dx=old.dx, level=1, origin=(old.origin[0] + 0.25, old.origin[1], old.origin[2]))
    with pytest.raises(ValueError):
        oracle.move_patch(par, _poly(par, 1), old, np.zeros(old.shape), bad)
    far = idd.Patch(n=old.n, dx=old.dx, level=1, origin=(old.origin[0] + 8.0, old.origin[1], old.origin[2]))
    with pytest.raises(ValueError):  # stencils leave the parent
        oracle.move_patch(par, _poly(par, 1), old, np.zeros(old.shape), far)


def _periodic_two_level(b):
    h = idd.Hierarchy(dx0=0.5, levels=[[idd.centred_patch(16, 0.5, level=0)],
                                       [idd.centred_patch(12, 0.25, centre=(0.5, 0.0, 0.0), level=1)]],
                      masses=[], positions=[])
    st = []
    for p in h.patches:
        u = idd.minkowski(p)
        for d in range(3):
            u[19 + d] = b[d]
        st.append(u)
    return h, st


def test_tracking_uniform_shift_exact():
    b = (0.3, -0.2, 0.1)
    h, st = _periodic_two_level(b)
    bo = oracle.BOHierarchy(h, st, oracle.Params(), courant=0.25, bc0=oracle.BC_PERIODIC)
    x0 = np.array([0.55, 0.05, -0.02])
    bo.track([x0], [-1, 0])
    for _ in range(3):
        bo.level_step(0)
    t = 3 * bo.dt(0)
    assert np.abs(bo.punct[0] - (x0 - np.array(b) * t)).max() < 1e-14


def test_tracking_heun_second_order():
    """Static linear shift beta^x = -a (x - xs): dx/dt = a (x - xs)."""
    a, xs, x0 = 0.8, 0.3, 0.6
    errs = []
    for courant in (0.4, 0.2, 0.1):
        h, st = _periodic_two_level((0.0, 0.0, 0.0))
        bo = oracle.BOHierarchy(h, st, oracle.Params(), courant=courant, bc0=oracle.BC_PERIODIC)
        p = bo.patches[1]
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        u = bo.tl[1][0].copy()
        u[19] = -a * (x - xs)
        bo.tl[1] = [u, u.copy()]
        bo.track([np.array([x0, 0.0, 0.0])], [-1, 0])
        nsteps = int(round(0.8 / bo.dt(1)))
        for _ in range(nsteps):
            bo._track(1)
        t = nsteps * bo.dt(1)
        errs.append(abs(bo.punct[0][0] - (xs + (x0 - xs) * math.exp(a * t))))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_regrid_recentres_and_nests():
    h = idd.moving_binary_3_level()
    st = idd.hierarchy_data(h)
    bo = oracle.BOHierarchy(h, st, oracle.Params(), courant=0.25)
    follow = [-1, 0, 1, 0, 1]
    bo.track(h.positions, follow)
    # move the punctures by hand (as if tracked): more than one parent cell
    bo.punct[0] = np.array([1.9, 0.6, 0.0])
    bo.punct[1] = np.array([-3.0, -1.55, 0.0])
    before = [bo.current(pid).copy() for pid in range(5)]
    old = list(bo.patches)
    moved = bo.regrid()
    assert moved >= 2
    for pid in range(1, 5):
        c = bo.patches[pid]
        for d in range(3):
            centre = c.origin[d] + 0.5 * c.n[d] * c.dx
            assert abs(bo.punct[follow[pid]][d] - centre) < 2 * c.dx + 1e-12
        lo, hi = bo.shift_range(pid)
        assert all(lo[d] <= 0 <= hi[d] for d in range(3))
        assert len(bo.tl[pid]) == 1
        # cells active before and after keep their values
        sh = [int(round((c.origin[d] - old[pid].origin[d]) / c.dx)) for d in range(3)]
        g, n = c.g, c.n
        sl_new = tuple(slice(g + max(0, -sh[d]), g + n[d] - max(0, sh[d])) for d in (2, 1, 0))
        sl_old = tuple(slice(g + max(0, sh[d]), g + n[d] - max(0, -sh[d])) for d in (2, 1, 0))
        assert np.array_equal(bo.current(pid)[(slice(None),) + sl_new], before[pid][(slice(None),) + sl_old])
    # a second regrid has nothing to do
    assert bo.regrid() == 0


def test_move_restarts_histories():
    """The moved patch's level always restarts its time-level history; the
    parent level only where its patches share active cells (the two level-1
    patches of this hierarchy overlap by 12 cells)."""
    h = idd.moving_binary_3_level()
    bo = oracle.BOHierarchy(h, idd.hierarchy_data(h), oracle.Params(), courant=0.5)
    bo.level_step(0)
    assert [len(bo.tl[i]) for i in range(5)] == [2, 3, 3, 3, 3]
    assert bo._active_overlap(1) and not bo._active_overlap(2)
    bo.move_patch(3, (1, 0, 0))
    assert [len(bo.tl[i]) for i in range(5)] == [2, 1, 1, 1, 1]
    bo.level_step(0)
    bo.move_patch(1, (-1, 0, 0))  # level 0 (one patch) keeps its history
    assert [len(bo.tl[i]) for i in range(5)] == [3, 1, 1, 3, 3]


def test_half_domain_shift_equals_full_domain():
    """Equatorial symmetry (Sec. 2.2.2) through a patch shift: the half-domain
    hierarchy that shifts a level-1 patch in x and y equals the upper half of
    the full-domain hierarchy doing the same on z-symmetric data."""
    h = idd.moving_binary_3_level()
    states = idd.hierarchy_data(h, noise=0.0)  # punctures on z = 0: symmetric
    for u in states:
        u[19] += 0.2   # a shift along x and y keeps the z symmetry
        u[20] -= 0.1
    hh = idd.upper_half_hierarchy(h)
    half = [idd.upper_half_array(p, u) for p, u in zip(h.patches, states)]
    full = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    half_bo = oracle.BOHierarchy(hh, half, oracle.Params(), courant=0.5, zsym=True)
    for bo in (full, half_bo):
        bo.level_step(0)
        bo.move_patch(1, (-1, 1, 0))
        bo.move_patch(4, (1, 0, 0))
        bo.level_step(0)
    with pytest.raises(ValueError):  # no z shifts under the symmetry
        half_bo.move_patch(3, (0, 0, 1))
    g = 3
    for i, p in enumerate(full.patches):
        a = idd.upper_half_array(p, full.current(i))[:, g:-g, g:-g, g:-g]
        b = half_bo.current(i)[:, g:-g, g:-g, g:-g]
        scale = np.maximum(np.abs(a).max(axis=(1, 2, 3)), 1e-300)
        assert (np.abs(a - b).max(axis=(1, 2, 3)) / scale).max() <= 1e-12, i
