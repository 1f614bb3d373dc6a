"""GPU parity of the fluid on the Berger-Oliger hierarchy (Sec. 2.2.1) with
the oracle (oracle/grhd_amr.py), through the C ABI, FP64: a periodic box
with a refined patch, the spacetime and a density wave evolved together,
the wave crossing the refinement boundary.  Both levels' primitives after
two coarse steps agree with the oracle's (conservative WENO5 ghost cells,
volume-averaged restriction, reflux), and the total rest mass of the
composite grid, computed from the GPU's state, is conserved to rounding."""
import math

import numpy as np
import pytest

import initial_data as idd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle
import paper_2607_08743_gb300 as sk
from oracle import grhd, grhd_amr as A
from paper_2607_08743_gb300 import build as skbuild

skbuild.build()

GAS = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)


def _setup(n0=24, nc=16, off=8):
    dx0 = 1.0 / n0
    P0 = idd.Patch(n=(n0, n0, n0), dx=dx0, origin=(-0.5, -0.5, -0.5), level=0)
    C1 = idd.Patch(n=(nc, nc, nc), dx=dx0 / 2, origin=tuple(-0.5 + off * dx0 for _ in range(3)), level=1)
    h = idd.Hierarchy(dx0=dx0, levels=[[P0], [C1]], masses=[], positions=[])
    v, W = 0.3, 1.0 / math.sqrt(1.0 - 0.09)

    def fluid(p):
        x = p.axis(0)
        pr = np.zeros((5,) + p.shape[1:])
        pr[0] = (1e-6 * (1.0 + 0.2 * np.sin(2.0 * np.pi * x)))[None, None, :]
        pr[1] = 1e-7 / ((5.0 / 3.0 - 1.0) * pr[0])
        pr[2] = W * v
        return pr
    return h, (P0, C1), fluid


def _rest_mass(ps, us, prims):
    cons = [grhd.prim2con(pr, grhd.metric(u), GAS)[0] for u, pr in zip(us, prims)]
    return A.rest_mass(list(ps), cons, [[1], []])


def test_two_level_fluid_matches_the_oracle_and_conserves_mass():
    h, ps, fluid = _setup()
    us = [idd.minkowski(p) for p in ps]
    prims = [fluid(p) for p in ps]
    g = sk.Grid(2, h.dx0, list(ps), sk.Params(matter=1, bc=1, lapse=1, shift=1, courant=0.25),
                stream=torch.cuda.Stream())
    g.set_eos(0.0, [2.0], (), 5.0 / 3.0)
    g.set_atmosphere(1e-18, 1e3)
    for i in range(2):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    H = A.MatterHierarchy(h, us, prims, GAS, [np.full(p.shape[1:], 1e-18) for p in ps],
                          oracle.Params(lapse=1, shift=1), courant=0.25, bc0=oracle.BC_PERIODIC)
    m0 = None
    for step in range(2):
        g.level_step(0)
        H.level_step(0)
        gu = [g.download_fields(i) for i in range(2)]
        gp = [g.download_matter(i) for i in range(2)]
        if m0 is None:
            m0 = _rest_mass(ps, us, prims)
        m = _rest_mass(ps, gu, gp)
        assert abs(m - m0) <= 1e-13 * m0, (step, (m - m0) / m0)
        for i, p in enumerate(ps):
            a = (slice(None),) + (slice(3, -3),) * 3
            want, got = H.prim(i)[a], gp[i][a]
            scale = np.maximum(np.abs(want - prims[i][a]).max(axis=(1, 2, 3)), 1e-3 * np.abs(want).max(axis=(1, 2, 3)))
            err = np.abs(got - want).max(axis=(1, 2, 3)) / scale
            assert err.max() <= 1e-9, (step, i, err)
    g.close()


def test_fluid_moves_need_an_uploaded_fluid_and_valid_followers():
    h, ps, fluid = _setup()
    g = sk.Grid(2, h.dx0, list(ps), sk.Params(matter=1, bc=1))
    with pytest.raises(sk.SacrakError):
        g.move_patch(1, (1, 0, 0))       # no fluid uploaded yet
    with pytest.raises(sk.SacrakError):
        g.density_maximum(0)
    with pytest.raises(sk.SacrakError):
        g.track_stars([0, -1])           # level 0 does not move
    with pytest.raises(sk.SacrakError):
        g.track_stars([-1, 1])           # star 0 followed by no patch
    g.close()
    s = sk.Grid(2, h.dx0, list(ps), sk.Params(bc=1))
    with pytest.raises(sk.SacrakError):
        s.track_stars([-1, 0])           # no fluid
    s.close()


def test_two_level_tov_star_matches_the_oracle():
    """A TOV star (R = 8.1 isotropic) on a 32^3 level (dx = 1) with a 32^3
    child (dx = 1/2) whose boundary at |x| = 8 crosses the star's surface:
    moving-puncture gauge, Sommerfeld ghosts on level 0, outflow fluid
    ghosts, atmosphere; two coarse steps against the oracle."""
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    P0 = idd.Patch(n=(32, 32, 32), dx=1.0, origin=(-16.0, -16.0, -16.0), level=0)
    C1 = idd.Patch(n=(32, 32, 32), dx=0.5, origin=(-8.0, -8.0, -8.0), level=1)
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
    g = sk.Grid(2, 1.0, [P0, C1], sk.Params(matter=1, courant=0.25), stream=torch.cuda.Stream())
    g.set_eos(star.K, [star.G], (), 1.8)
    g.set_atmosphere(1e-12 * 1.28e-3, 64.0)
    for i in range(2):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    H = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD)
    for _ in range(2):
        g.level_step(0)
        H.level_step(0)
    a = (slice(None),) + (slice(3, -3),) * 3
    errs = {}
    for i in range(2):
        ug, uo = g.download_fields(i)[a], H.current(i)[a]
        d = np.abs(ug - uo).max(axis=(1, 2, 3))
        # each field's change, floored at 1e-5 of its size (rounding of O(1)
        # fields that barely change on the coarse level)
        s = np.maximum(np.abs(uo - us[i][a]).max(axis=(1, 2, 3)), 1e-5 * np.abs(uo).max(axis=(1, 2, 3)) + 1e-12)
        pg, po = g.download_matter(i)[a], H.prim(i)[a]
        # velocities weighted by the density (in the tenuous atmosphere the
        # recovered velocity of tiny momenta is ill-conditioned)
        wt = po[0][None] / 1.28e-3
        errs[i] = ((d / s).max(), np.abs(pg[0] - po[0]).max() / 1.28e-3,
                   np.abs(wt * (pg[2:] - po[2:])).max() / max(np.abs(wt * po[2:]).max(), 1e-30))
    g.close()
    for i, (es, ed, ev) in errs.items():
        assert es <= 1e-9 and ed <= 1e-10 and ev <= 1e-9, errs


def _tov_hierarchy_data(patches, xc=0.0):
    """TOV star (R = 8.1 isotropic, centred at (xc, 0, 0)) data on the given
    patches: metric, primitives at rest on the cold curve, atmosphere
    floors."""
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
    us, prims, floors = [], [], []
    for p in patches:
        z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        rho, psi, al = star.fields(np.sqrt((x - xc) ** 2 + y * y + z * z))
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
    return star, eos, us, prims, floors


def _gpu_tov(patches, us, prims, star, zsym, steps):
    g = sk.Grid(len(patches), patches[0].dx, list(patches), sk.Params(matter=1, courant=0.25, zsym=int(zsym)),
                stream=torch.cuda.Stream())
    g.set_eos(star.K, [star.G], (), 1.8)
    g.set_atmosphere(1e-12 * 1.28e-3, 64.0)
    for i in range(len(patches)):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    for _ in range(steps):
        g.level_step(0)
    out = [(g.download_fields(i), g.download_matter(i)) for i in range(len(patches))]
    g.close()
    return out


def test_two_level_tov_star_equatorial_symmetry():
    """The two-level TOV star evolved on z >= 0 (equatorial symmetry, Sec.
    2.2.2; the fluid's and the spacetime's z < 0 ghosts reflected, the child
    on z = 0 prolonged from its parent's mirror image): two coarse steps
    against the oracle's half-domain hierarchy (same bounds as the full
    domain's test), and against the GPU's own full-domain evolution, whose
    upper half it reproduces to rounding."""
    P0 = idd.Patch(n=(32, 32, 32), dx=1.0, origin=(-16.0, -16.0, -16.0), level=0)
    C1 = idd.Patch(n=(32, 32, 32), dx=0.5, origin=(-8.0, -8.0, -8.0), level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    star, eos, us, prims, floors = _tov_hierarchy_data([P0, C1])
    hh = idd.upper_half_hierarchy(h)
    ph = hh.patches
    uh = [idd.upper_half_array(p, u) for p, u in zip((P0, C1), us)]
    prh = [idd.upper_half_array(p, a) for p, a in zip((P0, C1), prims)]
    flh = [idd.upper_half_array(p, f[None])[0] for p, f in zip((P0, C1), floors)]
    half = _gpu_tov(ph, uh, prh, star, True, 2)
    full = _gpu_tov((P0, C1), us, prims, star, False, 2)
    H = A.MatterHierarchy(hh, uh, prh, eos, flh, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD,
                          zsym=True)
    for _ in range(2):
        H.level_step(0)
    a = (slice(None),) + (slice(3, -3),) * 3
    errs = {}
    for i, p in enumerate((P0, C1)):
        (ug, pg), (uf, pf) = half[i], full[i]
        ug, pg = ug[a], pg[a]
        # the GPU's own full domain, upper half
        assert np.abs(ug - idd.upper_half_array(p, uf)[a]).max() <= 1e-13
        pfu = idd.upper_half_array(p, pf)[a]
        assert np.abs(pg[0] - pfu[0]).max() <= 1e-12 * 1.28e-3
        wf = pfu[0][None] / 1.28e-3  # eps and u_i weighted by the density, as below
        assert np.abs(wf * (pg[1:] - pfu[1:])).max() <= 1e-11 * np.abs(wf * pfu[1:]).max()
        # the oracle's half domain
        uo, po = H.current(i)[a], H.prim(i)[a]
        d = np.abs(ug - uo).max(axis=(1, 2, 3))
        s = np.maximum(np.abs(uo - uh[i][a]).max(axis=(1, 2, 3)), 1e-5 * np.abs(uo).max(axis=(1, 2, 3)) + 1e-12)
        wt = po[0][None] / 1.28e-3
        errs[i] = ((d / s).max(), np.abs(pg[0] - po[0]).max() / 1.28e-3,
                   np.abs(wt * (pg[2:] - po[2:])).max() / max(np.abs(wt * po[2:]).max(), 1e-30))
    for i, (es, ed, ev) in errs.items():
        assert es <= 1e-9 and ed <= 1e-10 and ev <= 1e-9, errs


def _bump(p):
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    pr = np.zeros((5,) + p.shape[1:])
    pr[0] = 1e-6 * (1.0 + 0.5 * np.exp(-((x - 0.05) ** 2 + y * y + z * z) / 0.02))
    pr[1] = 1e-7 / ((5.0 / 3.0 - 1.0) * pr[0])
    pr[2] = 0.1
    return pr


def test_moved_fluid_patch_matches_the_oracle_and_conserves_mass():
    """A smooth fluid bump on a periodic two-level box: a coarse step, the
    child shifted by (2, -1, 1) parent cells, another coarse step; both
    levels against the oracle's, and the composite rest mass from the GPU's
    state unchanged by the move."""
    h, ps, _ = _setup()
    us = [idd.minkowski(p) for p in ps]
    prims = [_bump(p) for p in ps]
    g = sk.Grid(2, h.dx0, list(ps), sk.Params(matter=1, bc=1, lapse=1, shift=1, courant=0.25),
                stream=torch.cuda.Stream())
    g.set_eos(0.0, [2.0], (), 5.0 / 3.0)
    g.set_atmosphere(1e-18, 1e3)
    for i in range(2):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    H = A.MatterHierarchy(h, us, prims, GAS, [np.full(p.shape[1:], 1e-18) for p in ps],
                          oracle.Params(lapse=1, shift=1), courant=0.25, bc0=oracle.BC_PERIODIC)
    g.level_step(0)
    H.level_step(0)

    def mass():
        gp = [g.download_matter(i) for i in range(2)]
        gu = [g.download_fields(i) for i in range(2)]
        geo = [ps[0], H.patches[1]]
        cons = [grhd.prim2con(pr, grhd.metric(u), GAS)[0] for u, pr in zip(gu, gp)]
        return A.rest_mass(geo, cons, [[1], []])
    g.move_patch(1, (2, -1, 1))
    H.move_patch(1, (2, -1, 1))
    assert g.patch_origin(1) == H.patches[1].origin
    m0 = H.rest_mass()
    assert abs(mass() - m0) <= 1e-13 * m0
    for stage in ("moved", "stepped"):
        for i in range(2):
            a = (slice(None),) + (slice(3, -3),) * 3
            want, got = H.prim(i)[a], g.download_matter(i)[a]
            scale = np.abs(want).max(axis=(1, 2, 3))
            err = np.abs(got - want).max(axis=(1, 2, 3)) / scale
            assert err.max() <= 1e-9, (stage, i, err)
        if stage == "moved":
            g.level_step(0)
            H.level_step(0)
    g.close()


def test_density_maximum_and_star_following_regrid():
    """A TOV star centred at x = 2.2 with the child centred on the origin:
    the density maximum against numpy on the GPU's own primitives, the
    star-following regrid's shift (2 parent cells, as the oracle's) and a
    coarse step after it against the oracle (the bounds of the unmoved
    TOV test)."""
    P0 = idd.Patch(n=(32, 32, 32), dx=1.0, origin=(-16.0, -16.0, -16.0), level=0)
    C1 = idd.Patch(n=(32, 32, 32), dx=0.5, origin=(-8.0, -8.0, -8.0), level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    from initial_data.tov import TOV
    star = TOV()
    eos = grhd.EOS(K0=star.K, gammas=[star.G], gamma_th=1.8)
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
    g = sk.Grid(2, 1.0, [P0, C1], sk.Params(matter=1, courant=0.25), stream=torch.cuda.Stream())
    g.set_eos(star.K, [star.G], (), 1.8)
    g.set_atmosphere(1e-12 * 1.28e-3, 64.0)
    for i in range(2):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    H = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD)
    g.track_stars([-1, 0])
    H.track_stars([-1, 0])
    g.level_step(0)
    H.level_step(0)
    for i, p in enumerate((P0, C1)):
        assert g.density_maximum(i) == A.density_maximum(p, g.download_matter(i))
    assert g.density_maximum(1)[1:] == H.star_positions()[0] == (2.25, -0.25, -0.25)
    assert g.regrid() == 1 and H.regrid() == 1
    assert g.patch_origin(1) == H.patches[1].origin == (-6.0, -8.0, -8.0)
    assert g.regrid() == 0
    g.level_step(0)
    H.level_step(0)
    a = (slice(None),) + (slice(3, -3),) * 3
    errs = {}
    for i in range(2):
        ug, uo = g.download_fields(i)[a], H.current(i)[a]
        d = np.abs(ug - uo).max(axis=(1, 2, 3))
        s = np.maximum(np.abs(uo - us[i][a]).max(axis=(1, 2, 3)), 1e-5 * np.abs(uo).max(axis=(1, 2, 3)) + 1e-12)
        pg, po = g.download_matter(i)[a], H.prim(i)[a]
        wt = po[0][None] / 1.28e-3
        errs[i] = ((d / s).max(), np.abs(pg[0] - po[0]).max() / 1.28e-3,
                   np.abs(wt * (pg[2:] - po[2:])).max() / max(np.abs(wt * po[2:]).max(), 1e-30))
    g.close()
    for i, (es, ed, ev) in errs.items():
        assert es <= 1e-9 and ed <= 1e-10 and ev <= 1e-9, errs


def test_star_following_under_equatorial_symmetry():
    """A TOV star at x = 2.2 on the upper half of the 32^3 two-level box
    (equatorial symmetry), the child following its density maximum: a coarse
    step, the regrid (2 parent cells along x), a coarse step, against the
    oracle's half-domain hierarchy (the unmoved TOV test's bounds)."""
    P0 = idd.Patch(n=(32, 32, 16), dx=1.0, origin=(-16.0, -16.0, 0.0), level=0)
    C1 = idd.Patch(n=(32, 32, 16), dx=0.5, origin=(-8.0, -8.0, 0.0), level=1)
    h = idd.Hierarchy(dx0=1.0, levels=[[P0], [C1]], masses=[], positions=[])
    star, eos, us, prims, floors = _tov_hierarchy_data([P0, C1], xc=2.2)
    g = sk.Grid(2, 1.0, [P0, C1], sk.Params(matter=1, courant=0.25, zsym=1), stream=torch.cuda.Stream())
    g.set_eos(star.K, [star.G], (), 1.8)
    g.set_atmosphere(1e-12 * 1.28e-3, 64.0)
    for i in range(2):
        g.upload_fields(i, us[i])
        g.upload_matter(i, prims[i])
    H = A.MatterHierarchy(h, us, prims, eos, floors, oracle.Params(), courant=0.25, bc0=oracle.BC_SOMMERFELD,
                          zsym=True)
    g.track_stars([-1, 0])
    H.track_stars([-1, 0])
    g.level_step(0)
    H.level_step(0)
    assert g.regrid() == 1 and H.regrid() == 1
    assert g.patch_origin(1) == H.patches[1].origin == (-6.0, -8.0, 0.0)
    g.level_step(0)
    H.level_step(0)
    a = (slice(None),) + (slice(3, -3),) * 3
    errs = {}
    for i in range(2):
        ug, uo = g.download_fields(i)[a], H.current(i)[a]
        d = np.abs(ug - uo).max(axis=(1, 2, 3))
        s = np.maximum(np.abs(uo - us[i][a]).max(axis=(1, 2, 3)), 1e-5 * np.abs(uo).max(axis=(1, 2, 3)) + 1e-12)
        pg, po = g.download_matter(i)[a], H.prim(i)[a]
        wt = po[0][None] / 1.28e-3
        errs[i] = ((d / s).max(), np.abs(pg[0] - po[0]).max() / 1.28e-3,
                   np.abs(wt * (pg[2:] - po[2:])).max() / max(np.abs(wt * po[2:]).max(), 1e-30))
    g.close()
    for i, (es, ed, ev) in errs.items():
        assert es <= 1e-9 and ed <= 1e-10 and ev <= 1e-9, errs
