"""Equatorial reflection symmetry of the fluid (Sec. 2.2.2: only z >= 0
evolved) in the oracle, pinned against the full domain: a TOV star on two
refinement levels evolved on the upper half with reflected ghosts equals
the upper half of the full-domain evolution, spacetime and fluid, to
rounding, and its rest-mass change is half the full domain's (no mass
crosses z = 0).  The reflection and the mirror extension used for a
child's prolongation are checked against brute force."""
import numpy as np
import pytest

import initial_data as idd
import oracle
from oracle import grhd, grhd_amr as A


def test_fluid_reflection_brute_force():
    p = idd.Patch(n=(6, 5, 4), dx=0.5, origin=(-1.0, -1.0, 0.0))
    rng = np.random.default_rng(5)
    g = p.g
    for parity, odd in ((A.PRIM_Z_PARITY, 4), (A.CONS_Z_PARITY, 3)):
        a = rng.normal(size=(5,) + p.shape[1:])
        b = A.fill_zreflect_fluid(p, a, parity)
        for f in range(5):
            sign = -1.0 if f == odd else 1.0  # u_z and J^_z are odd in z
            for k in range(g):
                assert np.array_equal(b[f, k], sign * a[f, 2 * g - 1 - k])
        assert np.array_equal(b[:, g:], a[:, g:])
        q, e = A.mirror_extend(p, b, parity, 2)
        assert q.n == (6, 5, 6) and q.origin == (-1.0, -1.0, -1.0)
        assert np.array_equal(e[:, 2:], b)
        for m in (1, 2):  # layer -m mirrors layer 2g - 1 + m
            assert np.array_equal(e[:, 2 - m], parity[:, None, None] * b[:, 2 * g - 1 + m])
    with pytest.raises(ValueError):
        A.fill_zreflect_fluid(idd.Patch(n=(4, 4, 4), dx=0.5, origin=(0, 0, 0.5)), np.zeros((5, 10, 10, 10)),
                              A.PRIM_Z_PARITY)


def _tov_two_levels(n0=24):
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    P0 = idd.Patch(n=(n0, n0, n0), dx=1.0, origin=(-n0 / 2,) * 3, level=0)
    C1 = idd.Patch(n=(n0, n0, n0), dx=0.5, origin=(-n0 / 4,) * 3, level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    us, prims, floors = [], [], []
    for p in (P0, C1):
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        rho, psi, al = star.fields(np.sqrt(x * x + y * y + z * z))
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
    return h, (P0, C1), eos, us, prims, floors


@pytest.fixture(scope="module")
def runs():
    """The star (R = 8.1) on a 24^3 level (dx = 1) and a 24^3 child (dx = 1/2,
    its boundary inside the star), one coarse step, full and half domain."""
    h, ps, eos, us, prims, floors = _tov_two_levels()
    full = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD)
    half = A.MatterHierarchy(idd.upper_half_hierarchy(h), [idd.upper_half_array(p, u) for p, u in zip(ps, us)],
                             [idd.upper_half_array(p, a) for p, a in zip(ps, prims)], eos,
                             [idd.upper_half_array(p, f[None])[0] for p, f in zip(ps, floors)],
                             oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD, zsym=True)
    m = (full.rest_mass(), half.rest_mass())
    full.level_step(0)
    half.level_step(0)
    return ps, us, full, half, m


def test_half_domain_equals_full_domain(runs):
    ps, us, full, half, _ = runs
    g = 3
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    for i, p in enumerate(ps):
        fu, hu = idd.upper_half_array(p, full.current(i))[a], half.current(i)[a]
        assert np.abs(fu - hu).max() <= 1e-14  # the spacetime's fields are O(1) or smaller
        assert np.abs(fu - idd.upper_half_array(p, us[i])[a]).max() > 1e-6  # and they moved
        fp, hp = idd.upper_half_array(p, full.prim(i))[a], half.prim(i)[a]
        scale = np.abs(fp).max(axis=(1, 2, 3))
        assert (np.abs(fp - hp).max(axis=(1, 2, 3)) <= 1e-12 * scale).all(), (i, np.abs(fp - hp).max(axis=(1, 2, 3)))


def test_half_domain_rest_mass_change_is_half_the_full(runs):
    """The atmosphere and the outflow boundary change the rest mass of both
    by 6e-12 of it; the half domain's change is exactly half the full one's."""
    _, _, full, half, (mf, mh) = runs
    assert abs(mf - 2.0 * mh) <= 1e-15 * mf
    df, dh = full.rest_mass() - mf, half.rest_mass() - mh
    assert abs(df - 2.0 * dh) <= 1e-15 * mf, (df, dh)
