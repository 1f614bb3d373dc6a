"""GPU parity of the matter sector (Sec. 2.1.2, 2.2) with the oracle
(oracle/grhd.py), through the C ABI, FP64:

* the conserved-variable right-hand side (PPM + face fluxes, geometric
  sources) on generic curved metric and fluid data and on a TOV star,
  ragged patch sizes included, with both face fluxes: HLLC in the face
  tetrad (the default) and HLLE in the coordinate frame;
* a contact discontinuity at rest, which HLLC keeps exactly;
* the recovery of the primitives with the atmosphere (cells below the floor
  reset to rest);
* the Z4c right-hand side with the fluid's terms;
* coupled RK4 steps of spacetime and fluid: TOV star with Sommerfeld ghosts
  and the moving-puncture gauge, generic data with frozen ghosts, and a
  density wave in a periodic box.

Tolerances: the two sides compute the same operations in a different order
(fused multiply-adds on the GPU), so values agree to rounding, 1e-11 of each
field's scale for single evaluations and 1e-9 after RK4 steps; the PPM
limiter's branch decisions take the same side except where their compared
quantities tie to rounding, which the smooth data here do not reach."""
import math

import numpy as np
import pytest

import initial_data as idd
import oracle
from oracle import grhd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

from tests import continuum as C

skbuild.build()

EOS = dict(K0=100.0, gammas=[2.0], gamma_th=1.8)


def _grid(p, **prm):
    g = sk.Grid(1, p.dx, [p], sk.Params(matter=1, **prm))
    g.set_eos(EOS["K0"], EOS["gammas"], (), EOS["gamma_th"])
    return g


def _eos():
    return grhd.EOS(K0=EOS["K0"], gammas=EOS["gammas"], gamma_th=EOS["gamma_th"])


def _rel(a, b, act=True):
    g = 3
    if act:
        a = a[:, g:-g, g:-g, g:-g]
        b = b[:, g:-g, g:-g, g:-g]
    scale = np.abs(b).max(axis=(1, 2, 3))
    return np.abs(a - b).max(axis=(1, 2, 3)) / np.where(scale > 0, scale, 1.0)


def _generic(n):
    """The curved generic metric of the continuum pins and a generic fluid on
    an n^3 patch (the fluid scaled to the EOS of this module)."""
    p, pts, u = C.patch_state(n)
    prim = np.ascontiguousarray(C.on_points(C.fluid_prims, pts).T.reshape((5,) + p.shape[1:]))
    return p, u, prim


def _tov(n, half=12.0):
    from initial_data.tov import TOV
    star = TOV()
    p = idd.centred_patch(n, 2 * half / n)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    rho, psi, al = star.fields(np.sqrt(x * x + y * y + z * z))
    u = idd.minkowski(p)
    u[0] = psi ** -2
    u[18] = al
    floor = grhd.atmosphere_floor(p, 1.28e-3, 1e-12, 8 * 2 * half)
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = np.maximum(rho, floor)
    prim[1] = _eos().cold(prim[0])[1]
    return p, u, prim, floor


def _oracle_state(p, u, prim, floor, periodic=False):
    eos = _eos()
    cons, _, _, _ = grhd.prim2con(prim, grhd.metric(u), eos)
    pr, cons, _ = grhd.recover(cons, u, eos, floor)
    pr = (grhd.periodic_ghosts if periodic else grhd.outflow_ghosts)(p, pr)
    return cons, pr


def _upload(g, u, prim, rho_atm, r_atm):
    g.set_atmosphere(rho_atm, r_atm)
    g.upload_fields(0, u)
    g.upload_matter(0, prim)


@pytest.mark.parametrize("solver", ["hllc", "hlle"])
@pytest.mark.parametrize("n", [(16, 16, 16), (18, 12, 10)])
def test_matter_rhs_generic(n, solver):
    p0, u0, prim0 = _generic(32)  # the ragged patch is cut from the 32^3 data
    p = idd.Patch(n=n, dx=p0.dx, origin=p0.origin)
    sl = (slice(None), slice(0, n[2] + 6), slice(0, n[1] + 6), slice(0, n[0] + 6))
    u = np.ascontiguousarray(u0[sl])
    prim = np.ascontiguousarray(prim0[sl])
    floor = np.full(p.shape[1:], 1e-12 * 3e-3)
    g = _grid(p, bc=2)
    g.set_riemann(solver)
    _upload(g, u, prim, 1e-12 * 3e-3, 1e3)
    r = g.matter_rhs(0)
    cons, pr = _oracle_state(p, u, prim, floor)
    ro = grhd.matter_rhs(p, pr, u, _eos(), solver=solver)
    e = _rel(r, ro)
    assert e.max() <= 1e-11, e
    assert np.all(r[:, :3] == 0.0) and np.all(r[:, :, :, -3:] == 0.0)
    # the recovered primitives
    np.testing.assert_allclose(g.download_matter(0)[:, 3:-3, 3:-3, 3:-3], pr[:, 3:-3, 3:-3, 3:-3], rtol=1e-12,
                               atol=1e-15)
    g.close()


@pytest.mark.parametrize("solver", ["hllc", "hlle"])
def test_matter_rhs_tov(solver):
    p, u, prim, floor = _tov(32)
    g = _grid(p, bc=0)
    g.set_riemann(solver)
    _upload(g, u, prim, 1e-12 * 1.28e-3, 8 * 24.0)
    r = g.matter_rhs(0)
    cons, pr = _oracle_state(p, u, prim, floor)
    ro = grhd.matter_rhs(p, pr, u, _eos(), solver=solver)
    # at rest D and E fluxes are numerical dissipation only: scale per field
    e = _rel(r, ro)
    assert e.max() <= 1e-10, e
    g.close()


def test_atmosphere_reset_matches_oracle():
    """Cells below the floor density (and one with no physical root) come back
    at rest on the cold curve at the floor."""
    p, u, prim = _generic(16)
    prim = prim.copy()
    prim[0, 8:11, 5:9, 4:12] = 1e-20
    floor = np.full(p.shape[1:], 1e-9)
    g = _grid(p, bc=2)
    _upload(g, u, prim, 1e-9, 1e3)
    g.matter_rhs(0)  # recovers (and resets) the current state
    got = g.download_matter(0)
    cons, pr = _oracle_state(p, u, prim, floor)
    a = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    np.testing.assert_allclose(got[a], pr[a], rtol=1e-12, atol=1e-15)
    assert np.all(got[0, 8:11, 5:9, 4:12] == 1e-9) and np.all(got[2:, 8:11, 5:9, 4:12] == 0.0)
    g.close()


def test_z4c_rhs_with_matter_terms():
    p, u, prim = _generic(16)
    floor = np.full(p.shape[1:], 1e-12 * 3e-3)
    g = _grid(p, bc=2)
    _upload(g, u, prim, 1e-12 * 3e-3, 1e3)
    r = g.rhs(0)
    cons, pr = _oracle_state(p, u, prim, floor)
    ro = oracle.rhs(p, u, oracle.Params()) + grhd.z4c_matter_rhs(pr, u, _eos())
    e = _rel(r, ro)
    assert e.max() <= 1e-12, dict(zip(idd.FIELD_NAMES, e))
    g.close()


def _steps(p, u, prim, floor, rho_atm, r_atm, steps, bc, gprm):
    dt = 0.25 * p.dx
    g = _grid(p, bc={"sommerfeld": 0, "periodic": 1, "frozen": 2}[bc], **gprm)
    _upload(g, u, prim, rho_atm, r_atm)
    eos = _eos()
    cons, _ = _oracle_state(p, u, prim, floor, periodic=bc == "periodic")
    uo = u
    prm = oracle.Params(**{k: v for k, v in gprm.items() if k in ("shift", "lapse")})
    for _ in range(steps):
        g.rk4_step(0, dt)
        uo, cons, pro = grhd.rk4_step_coupled(p, uo, cons, dt, eos, floor, prm, bc=bc)
    ug, pg = g.download_fields(0), g.download_matter(0)
    g.close()
    return ug, pg, uo, pro


def _change_err(v, vo, v0, floor=0.0):
    g = 3
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    d = np.abs(v[a] - vo[a]).max(axis=(1, 2, 3))
    s = np.maximum(np.abs(vo[a] - v0[a]).max(axis=(1, 2, 3)), floor)
    return d / np.where(s > 0, s, 1.0)


def test_coupled_steps_tov():
    """Two RK4 steps of the TOV star with the 1+log / Gamma-driver gauge and
    Sommerfeld ghosts: spacetime and fluid against the oracle."""
    p, u, prim, floor = _tov(32)
    ug, pg, uo, pro = _steps(p, u, prim, floor, 1e-12 * 1.28e-3, 8 * 24.0, 2, "sommerfeld", {})
    e = _change_err(ug, uo, u)
    assert e.max() <= 1e-9, dict(zip(idd.FIELD_NAMES, e))
    a = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    # the density changes little; compare on the density scale
    np.testing.assert_allclose(pg[0][a[1:]], pro[0][a[1:]], rtol=0, atol=1e-10 * 1.28e-3)
    np.testing.assert_allclose(pg[2:][a], pro[2:][a], rtol=0, atol=1e-9 * max(np.abs(pro[2:][a]).max(), 1e-12))


def test_coupled_step_generic_frozen_ghosts():
    p, u, prim = _generic(16)
    floor = np.full(p.shape[1:], 1e-12 * 3e-3)
    ug, pg, uo, pro = _steps(p, u, prim, floor, 1e-12 * 3e-3, 1e3, 1, "frozen", {})
    e = _change_err(ug, uo, u)
    assert e.max() <= 1e-9, dict(zip(idd.FIELD_NAMES, e))
    em = _change_err(pg, pro, prim)
    assert em.max() <= 1e-9, em


def test_coupled_steps_density_wave_periodic():
    """A density wave (rho ~ 1e-6, so the spacetime barely responds) advected
    with uniform velocity in a periodic box, frozen shift, harmonic lapse."""
    n = 32
    dx = 1.0 / n
    p = idd.Patch(n=(n, 4, 4), dx=dx, origin=(-0.5, -2 * dx, -2 * dx))
    u = idd.minkowski(p)
    x = p.axis(0)
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = (1e-6 * (1.0 + 0.2 * np.sin(2 * np.pi * x)))[None, None, :]
    prim[1] = 0.2
    prim[2] = 0.3 / math.sqrt(1 - 0.09)
    floor = np.full(p.shape[1:], 1e-18)
    ug, pg, uo, pro = _steps(p, u, prim, floor, 1e-18, 1e3, 4, "periodic", {"shift": 1, "lapse": 1})
    e = _change_err(ug, uo, u, floor=1e-12)
    assert e.max() <= 1e-9, dict(zip(idd.FIELD_NAMES, e))
    em = _change_err(pg, pro, prim)
    assert em[0] <= 1e-9 and em[2] <= 1e-9, em


def test_contact_at_rest_is_stationary_with_hllc():
    """A density step at rest with uniform pressure on flat space: HLLC in the
    face tetrad resolves the contact, so the fluid's right-hand side is zero
    to rounding; with HLLE the density diffuses."""
    n = 16
    p = idd.centred_patch(n, 1.0 / n)
    u = idd.minkowski(p)
    gas = dict(K0=0.0, gammas=[2.0], gamma_th=5.0 / 3.0)
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = np.where(np.abs(p.axis(0)) < 0.25, 2.0, 1.0)[None, None, :]
    prim[1] = 1.0 / ((5.0 / 3.0 - 1.0) * prim[0])
    out = {}
    for solver in ("hllc", "hlle"):
        g = sk.Grid(1, p.dx, [p], sk.Params(matter=1, bc=1))
        g.set_eos(gas["K0"], gas["gammas"], (), gas["gamma_th"])
        g.set_riemann(solver)
        _upload(g, u, prim, 1e-12, 1e3)
        out[solver] = g.matter_rhs(0)
        g.close()
    assert np.abs(out["hllc"][[0, 2, 3, 4]]).max() <= 1e-13
    assert np.abs(out["hllc"][1]).max() <= 1e-12
    assert np.abs(out["hlle"][0]).max() > 1e-2


def test_matter_arguments_rejected():
    p = idd.centred_patch(8, 1.0)
    g = sk.Grid(1, p.dx, [p], sk.Params())
    with pytest.raises(sk.SacrakError):
        g.set_eos(100.0, [2.0])          # grid without a fluid
    g.close()
    m = _grid(p)
    with pytest.raises(sk.SacrakError):
        m.rk4_step(0)                    # no fluid uploaded yet
    with pytest.raises(sk.SacrakError):
        m.set_eos(100.0, [0.9])          # index <= 1
    with pytest.raises(sk.SacrakError):
        m.set_atmosphere(-1.0, 1.0)
    with pytest.raises(sk.SacrakError):
        m._check(sk.lib().sacrak_set_riemann(m._h, 2), "set_riemann")
    with pytest.raises(sk.SacrakError):
        m.upload_matter(0, np.zeros((5, 3, 3, 3)))
    m.close()
    with pytest.raises(sk.SacrakError):  # a fluid needs one FP64 level
        sk.Grid(1, p.dx, [p], sk.Params(matter=1, precision=1))


@pytest.mark.parametrize("solver", ["hllc", "hlle"])
def test_blast_wave_tube_against_oracle(solver):
    """The relativistic blast wave (left rho = 10, P = 13.33, right rho = 1,
    P = 1e-6, ideal gas Gamma = 5/3, at rest) scaled by 1e-8 in density and
    pressure (the Riemann problem is unchanged; the spacetime barely
    responds), 16 RK4 steps on a 64-cell tube with Sommerfeld ghosts: the
    shock, the contact and the rarefaction form, and the fluid agrees with
    the oracle to 1e-9 of its scale.  The spacetime's response (about 1e-8)
    agrees to 1e-5 of itself: the two round the O(1) metric fields
    differently at about 1e-15."""
    n, s = 64, 1e-8
    dx = 1.0 / n
    p = idd.Patch(n=(n, 4, 4), dx=dx, origin=(-0.5, -2 * dx, -2 * dx))
    u = idd.minkowski(p)
    x = p.axis(0)
    gam = 5.0 / 3.0
    prim = np.zeros((5,) + p.shape[1:])
    prim[0] = np.where(x < 0, 10.0 * s, 1.0 * s)[None, None, :]
    prim[1] = np.where(x < 0, 13.33 / 10.0, 1e-6)[None, None, :] / (gam - 1.0)
    floor = np.full(p.shape[1:], 1e-20)
    eos = grhd.EOS(K0=0.0, gammas=[2.0], gamma_th=gam)
    g = sk.Grid(1, p.dx, [p], sk.Params(matter=1, bc=0))
    g.set_eos(0.0, [2.0], (), gam)
    g.set_riemann(solver)
    _upload(g, u, prim, 1e-20, 1e3)
    cons, _, _, _ = grhd.prim2con(prim, grhd.metric(u), eos)
    uo, dt = u, 0.25 * dx
    for _ in range(16):
        g.rk4_step(0, dt)
        uo, cons, pro = grhd.rk4_step_coupled(p, uo, cons, dt, eos, floor, oracle.Params(), solver=solver)
    ug, pg = g.download_fields(0), g.download_matter(0)
    g.close()
    a = (slice(3, -3), slice(3, -3), slice(3, -3))
    right = np.flatnonzero(x[3:-3] > 0)
    assert pro[0][a][..., right].max() > 2.0 * s  # the compressed shell behind the shock
    assert pro[2][a].max() > 0.5  # the flow reaches W v ~ 1 behind the contact
    np.testing.assert_allclose(pg[0][a], pro[0][a], rtol=0, atol=1e-9 * 10.0 * s)
    np.testing.assert_allclose(pg[1][a], pro[1][a], rtol=0, atol=1e-9 * np.abs(pro[1][a]).max())
    np.testing.assert_allclose(pg[2:][(slice(None),) + a], pro[2:][(slice(None),) + a], rtol=0, atol=1e-9)
    e = _change_err(ug, uo, u, floor=1e-14)
    assert e.max() <= 1e-5, dict(zip(idd.FIELD_NAMES, e))
