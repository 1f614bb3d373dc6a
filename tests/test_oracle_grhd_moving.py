"""Moving patches with a fluid in the oracle (Sec. 2.2.1: a neutron star is
located by its rest-mass density maximum, its patches shift in steps of two
cells, newly covered cells are prolonged from the parent).

* The density maximum against brute force (ties: the first cell in z, y, x
  order).
* A move conserves the total rest mass of the composite grid to rounding
  (a smooth positive fluid, after a coarse step's restriction): cells
  active before and after keep their values, newly covered cells take the
  conservative WENO5 prolongation of D^ (the 8 children of a parent cell
  average to it), uncovered parent cells hold the restriction of the old
  child.  Cell by cell: the copied block is bitwise the old one, the new
  block averages to the parent.
* A uniform fluid stays uniform through a move.
* Star following: a TOV star off the child's centre; regrid() moves the
  child by trunc(offset / dx_parent) parent cells toward the density
  maximum, and the evolution continues."""

import numpy as np
import pytest

import initial_data as idd
import oracle
from oracle import grhd, grhd_amr as A

GAS = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)


def test_density_maximum_brute_force():
    p = idd.Patch(n=(7, 6, 5), dx=0.5, origin=(-1.0, 2.0, 0.5))
    rng = np.random.default_rng(9)
    prim = rng.random((5,) + p.shape[1:])
    g = p.g
    prim[0, g + 3, g + 2, g + 4] = 2.0
    prim[0, g + 4, g + 1, g + 1] = 2.0  # a tie later in z: the first one wins
    prim[0, 0, 0, 0] = 5.0              # ghosts do not count
    r, x, y, z = A.density_maximum(p, prim)
    assert r == 2.0 and (x, y, z) == (-1.0 + 4.5 * 0.5, 2.0 + 2.5 * 0.5, 0.5 + 3.5 * 0.5)


def test_lagrange_children_exact_for_quintics_and_matches_the_ghost_operator():
    """The all-cells 6th-order Lagrange prolongation used by moves: exact on a
    quintic in x, y and z (cell centres), and on the ghost shell the same
    values as the ghost prolongation (the C oracle's, tensor product)."""
    P = idd.Patch(n=(16, 16, 16), dx=1.0, origin=(-8.0,) * 3, level=0)
    C = idd.Patch(n=(8, 8, 8), dx=0.5, origin=(-2.0, -1.0, -3.0), level=1)
    def quint(p):
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        return 0.3 * x ** 5 - 0.1 * y ** 4 * x + 0.05 * z ** 5 + 0.2 * x * y * z + 1.0
    q = quint(P)
    got = A.lagrange_prolong_cells(P, C, q)
    want = quint(C)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    rng = np.random.default_rng(4)
    r = rng.random(P.shape[1:])
    m = A.ghost_mask(C)
    a = A.lagrange_prolong_cells(P, C, r)[m]
    b = A.lagrange_prolong(P, C, [r])[0][m]
    assert np.abs(a - b).max() <= 1e-14


def _smooth_hierarchy(fluid_fn):
    n0, nc, off = 24, 16, 8
    dx0 = 1.0 / n0
    P0 = idd.Patch(n=(n0, n0, n0), dx=dx0, origin=(-0.5, -0.5, -0.5), level=0)
    C1 = idd.Patch(n=(nc, nc, nc), dx=dx0 / 2, origin=tuple(-0.5 + off * dx0 for _ in range(3)), level=1)
    h = idd.Hierarchy(dx0=dx0, levels=[[P0], [C1]], masses=[], positions=[])
    ps = (P0, C1)
    return A.MatterHierarchy(h, [idd.minkowski(p) for p in ps], [fluid_fn(p) for p in ps], GAS,
                             [np.full(p.shape[1:], 1e-18) for p in ps], oracle.Params(lapse=1, shift=1),
                             courant=0.25, bc0=oracle.BC_PERIODIC)


def _bump(p):
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    pr = np.zeros((5,) + p.shape[1:])
    pr[0] = 1e-6 * (1.0 + 0.5 * np.exp(-((x - 0.05) ** 2 + y * y + z * z) / 0.02))
    pr[1] = 1e-7 / ((5.0 / 3.0 - 1.0) * pr[0])
    pr[2] = 0.1
    return pr


def test_move_conserves_rest_mass():
    H = _smooth_hierarchy(_bump)
    H.level_step(0)
    m0 = H.rest_mass()
    P, C = H.patches
    g = 3
    old = H.cons(1)[:, g:-g, g:-g, g:-g].copy()
    H.move_patch(1, (2, -1, 1))
    C2 = H.patches[1]
    assert C2.origin == tuple(C.origin[d] + 2 * s * C.dx for d, s in enumerate((2, -1, 1)))
    assert abs(H.rest_mass() - m0) <= 1e-14 * m0, (H.rest_mass() - m0) / m0
    new = H.cons(1)[:, g:-g, g:-g, g:-g]
    # the block active before and after: new cell i is old cell i + (4, -2, 2)
    assert np.array_equal(new[:, 0:14, 2:16, 0:12], old[:, 2:16, 0:14, 4:16])
    # every child block averages to its parent cell (copied blocks: the restriction)
    off = A.child_offset(P, C2)
    Dp = H.cons(0)[0, g:-g, g:-g, g:-g][off[2]:off[2] + 8, off[1]:off[1] + 8, off[0]:off[0] + 8]
    mean = new[0].reshape(8, 2, 8, 2, 8, 2).mean(axis=(1, 3, 5))
    assert np.abs(mean - Dp).max() <= 1e-15 * np.abs(Dp).max()
    H.level_step(0)  # and it evolves on
    assert np.isfinite(H.prim(1)).all()


def test_uniform_fluid_stays_uniform_through_a_move():
    def uniform(p):
        pr = np.zeros((5,) + p.shape[1:])
        pr[0], pr[1], pr[2], pr[3], pr[4] = 2e-6, 0.4, 0.1, -0.2, 0.05
        return pr
    H = _smooth_hierarchy(uniform)
    H.move_patch(1, (-3, 2, 0))
    g = 3
    pr = H.prim(1)
    for f, want in enumerate([2e-6, 0.4, 0.1, -0.2, 0.05]):
        assert np.abs(pr[f] - want).max() <= 1e-14 * abs(want)


def test_star_following_regrid():
    """A TOV star centred at x = 2.2 in a two-level box whose child is
    centred on the origin: after a coarse step the density maximum is the
    cell at x = 2.25, and regrid() shifts the child by trunc(2.25 / 1) = 2
    parent cells (its nesting allows up to 2); a further coarse step runs."""
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    P0 = idd.Patch(n=(24, 24, 24), dx=1.0, origin=(-12.0,) * 3, level=0)
    C1 = idd.Patch(n=(24, 24, 24), dx=0.5, origin=(-6.0,) * 3, level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    us, prims, floors = [], [], []
    for p in (P0, C1):
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        rho, psi, al = star.fields(np.sqrt((x - 2.2) ** 2 + y * y + z * z))
        u = idd.minkowski(p)
        u[0] = psi ** -2
        u[18] = al
        fl = grhd.atmosphere_floor(p, 1.28e-3, 1e-12, 64.0)
        pr = np.zeros((5,) + p.shape[1:])
        pr[0] = np.maximum(rho, fl)
        pr[1] = eos.cold(pr[0])[1]
        us.append(u)
        prims.append(pr)
        floors.append(fl)
    H = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD)
    H.track_stars([-1, 0])
    with pytest.raises(ValueError):
        H.track_stars([0, -1])  # level 0 does not move
    H.level_step(0)
    r, x, y, z = A.density_maximum(H.patches[1], H.prim(1))
    assert (x, y, z) == (2.25, -0.25, -0.25) and r > 1e-3
    assert H.star_positions() == {0: (2.25, -0.25, -0.25)}
    assert H.regrid() == 1
    assert H.patches[1].origin == (-4.0, -6.0, -6.0)
    assert H.regrid() == 0  # the star now lies within a parent cell of the centre
    H.level_step(0)
    assert np.isfinite(H.prim(1)).all() and np.isfinite(H.current(1)).all()


def test_star_following_under_equatorial_symmetry_equals_full_domain():
    """The star-following run above on the upper half (equatorial symmetry:
    no shift along z, the moved child's z < 0 ghosts reflected) equals the
    upper half of the full-domain run: a coarse step, the regrid, and a
    coarse step after it."""
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    P0 = idd.Patch(n=(24, 24, 24), dx=1.0, origin=(-12.0,) * 3, level=0)
    C1 = idd.Patch(n=(24, 24, 24), dx=0.5, origin=(-6.0,) * 3, level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    us, prims, floors = [], [], []
    for p in (P0, C1):
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        rho, psi, al = star.fields(np.sqrt((x - 2.2) ** 2 + y * y + z * z))
        u = idd.minkowski(p)
        u[0] = psi ** -2
        u[18] = al
        fl = grhd.atmosphere_floor(p, 1.28e-3, 1e-12, 64.0)
        pr = np.zeros((5,) + p.shape[1:])
        pr[0] = np.maximum(rho, fl)
        pr[1] = eos.cold(pr[0])[1]
        us.append(u)
        prims.append(pr)
        floors.append(fl)
    ps = (P0, C1)
    full = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD)
    half = A.MatterHierarchy(idd.upper_half_hierarchy(h), [idd.upper_half_array(p, u) for p, u in zip(ps, us)],
                             [idd.upper_half_array(p, a) for p, a in zip(ps, prims)], eos,
                             [idd.upper_half_array(p, f[None])[0] for p, f in zip(ps, floors)],
                             oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD, zsym=True)
    for H in (full, half):
        H.track_stars([-1, 0])
        H.level_step(0)
    # the full domain's maximum may sit just below z = 0 (cells at z = +-0.25
    # hold equal densities): only x decides the shift here
    assert full.regrid() == 1 and half.regrid() == 1
    assert full.patches[1].origin[:2] == half.patches[1].origin[:2] == (-4.0, -6.0)
    assert half.patches[1].origin[2] == 0.0
    full.level_step(0)
    half.level_step(0)
    g = 3
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    for i in range(2):
        pf, ph = full.patches[i], half.patches[i]
        fu = idd.upper_half_array(pf, full.current(i))[a]
        assert np.abs(fu - half.current(i)[a]).max() <= 1e-14
        fp, hp = idd.upper_half_array(pf, full.prim(i))[a], half.prim(i)[a]
        assert np.abs(fp[0] - hp[0]).max() <= 1e-13 * 1.28e-3
        # eps and u_i weighted by the density (in the atmosphere the values
        # recovered from tiny conserved variables are ill-conditioned)
        wt = fp[0][None] / 1.28e-3
        assert np.abs(wt * (fp[1:] - hp[1:])).max() <= 1e-12 * np.abs(wt * fp[1:]).max()
