"""Pins of the oracle's Theta-coupled and constraint-damping terms of the Z4c
right-hand side (Sec. 2.1.1: Z4c with the damping terms applied locally;
Sec. 3: kappa1 = 0.005/M, kappa2 = 0).

The continuum pin (test_oracle_continuum.py) runs with Theta = 0 and the
evolved Gamt^i equal to Gamd^i, where these terms vanish.  Here every term
that carries Theta, kappa1 or kappa2 is isolated by linearity and compared
with a value computed by another route:

* kappa1, kappa2 enter only through the damping terms, so the difference of
  two right-hand sides of the same state with different (kappa1, kappa2) is
  exactly the damping part.  Its Khat and Theta parts are derived here from
  the damped Z4 system in 3+1 form (Gundlach et al. 2005: d_t K_ij gets
  -alpha kappa1 (1+kappa2) Theta gamma_ij, d_t Theta gets
  -alpha kappa1 (2+kappa2) Theta), with Khat = gamma^ij K_ij - 2 Theta; the
  Gamt part is the Z4c form -2 alpha kappa1 (Gamt^i - Gamd^i) with Gamd^i =
  -d_j gt^ij taken from autograd of the analytic metric.
* Moving Theta into Khat at fixed K = Khat + 2 Theta leaves every K-term
  unchanged, so the difference isolates the damping terms and the d_j Theta
  term of the Gamt equation, 2 alpha gt^ij d_j theta for Theta -> Theta +
  theta, Khat -> Khat - 2 theta.
* For spatially constant data every derivative vanishes exactly, and the
  right-hand side is the algebraic part of the equations, computed here
  from the physical K_ij and gamma_ij.

A dropped lapse factor, 2 - kappa2 for 2 + kappa2, a wrong factor on
d_j Theta, or Khat in place of Khat + 2 Theta inside K fails one of them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import initial_data as idd
import oracle

from tests import continuum as C

KH, TH, ALP = 7, 8, 18
GAM = [15, 16, 17]
BV = [22, 23, 24]
DAMPED = [KH, TH] + GAM + BV


def _sample(p):
    g = p.g
    st = max(p.n[0] // 8, 1)
    return slice(g, g + p.n[0], st)


def _at(p, a):
    s = _sample(p)
    return a[..., s, s, s]


def _sample_points(p):
    s = _sample(p)
    z, y, x = np.meshgrid(p.axis(2)[s], p.axis(1)[s], p.axis(0)[s], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _field(fn, pts, shape):
    return C.on_points(fn, pts).reshape(shape)


def _damped_state(n):
    """Generic data with Theta = theta(x) and Gamt^i = Gamd^i + c^i(x)."""
    p, pts, u0 = C.patch_state(n)
    u = u0.copy()
    u[TH] = _field(C.theta, pts, p.shape[1:])
    off = C.on_points(C.gam_offset, pts).T.reshape((3,) + p.shape[1:])
    for i in range(3):
        u[GAM[i]] += off[i]
    return p, u


def _gamd_sample(p):
    """Gamd^i = -d_j gt^ij of the analytic metric (det gt = 1) at the sample."""
    return C.on_points(C.Gamt_of, _sample_points(p)).T


@pytest.mark.parametrize("k1,k2", [(0.4, 0.0), (0.4, 0.3), (0.25, -0.5), (0.005, 0.0)])
def test_damping_terms_by_kappa_difference(k1, k2):
    """rhs(kappa1, kappa2) - rhs(0, 0) on generic data (full right-hand side:
    advection and dissipation cancel in the difference).  Khat, Theta:
    exactly the Z4-derived damping (to rounding); Gamt, B: the Z4c damping of
    Gamt - Gamd (Gamd discrete, so to truncation: 4th order in h); every
    other field: exactly zero."""
    errs = {}
    for n in (16, 32):
        p, u = _damped_state(n)
        r1 = oracle.rhs(p, u, oracle.Params(kappa1=k1, kappa2=k2))
        r0 = oracle.rhs(p, u, oracle.Params(kappa1=0.0, kappa2=0.0))
        d = _at(p, r1 - r0)
        scale = np.abs(_at(p, r1)).max()
        a, th = _at(p, u[ALP]), _at(p, u[TH])
        # damped Z4 in 3+1 form: d_t K_ij -= alpha k1 (1+k2) Theta gamma_ij,
        # d_t Theta -= alpha k1 (2+k2) Theta; Khat = gamma^ij K_ij - 2 Theta
        dK = -a * k1 * (1.0 + k2) * th * 3.0  # gamma^ij gamma_ij = 3
        dTh = -a * k1 * (2.0 + k2) * th
        np.testing.assert_allclose(d[TH], dTh, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(d[KH], dK - 2.0 * dTh, rtol=0, atol=1e-13 * scale)
        for f in range(25):
            if f not in DAMPED:
                assert np.all(d[f] == 0.0), idd.FIELD_NAMES[f]
        gd = _gamd_sample(p).reshape((3,) + d.shape[1:])
        e, exmax = 0.0, 0.0
        for i in range(3):
            ex = -2.0 * a * k1 * (_at(p, u[GAM[i]]) - gd[i])
            e = max(e, np.abs(d[GAM[i]] - ex).max())
            exmax = max(exmax, np.abs(ex).max())
            # B^i carries the same Gamt source (Gamma driver)
            np.testing.assert_allclose(d[BV[i]], d[GAM[i]], rtol=0, atol=1e-13 * scale)
        assert exmax > 0.02 * k1
        errs[n] = e / exmax
    # relative to the term (O(k1 * 0.05)): the truncation error of the
    # discrete Gamd (4th-order stencils) falls at 4th order
    assert errs[32] < 2e-4, errs
    assert np.log2(errs[16] / errs[32]) > 3.5, errs


@pytest.mark.parametrize("k1,k2", [(0.3, 0.2), (0.3, 0.0)])
def test_theta_shift_at_fixed_K(k1, k2):
    """Theta -> Theta + theta, Khat -> Khat - 2 theta (K = Khat + 2 Theta
    unchanged), sources only.  W, gt, At, alpha (1+log with K), beta: no
    change; Khat, Theta: the damping of theta; Gamt, B: 2 alpha gt^ij d_j theta
    from the -2/3 alpha gt^ij (2 d_j Khat + d_j Theta) term, to 4th order."""
    errs = {}
    for n in (16, 32):
        p, pts, u1 = C.patch_state(n)
        th = _field(C.theta, pts, p.shape[1:])
        u2 = u1.copy()
        u2[TH] += th
        u2[KH] -= 2.0 * th
        prm = oracle.Params(kappa1=k1, kappa2=k2)
        r1 = oracle.rhs(p, u1, prm, terms=1)
        r2 = oracle.rhs(p, u2, prm, terms=1)
        d = _at(p, r2 - r1)
        scale = np.abs(_at(p, r1)).max()
        a, ts = _at(p, u1[ALP]), _at(p, th)
        for f in [0, 1, 2, 3, 4, 5, 6, 9, 10, 11, 12, 13, 14, ALP, 19, 20, 21]:
            np.testing.assert_allclose(d[f], 0.0, rtol=0, atol=1e-13 * scale, err_msg=idd.FIELD_NAMES[f])
        np.testing.assert_allclose(d[KH], a * k1 * (1.0 - k2) * ts, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(d[TH], -a * k1 * (2.0 + k2) * ts, rtol=0, atol=1e-13 * scale)
        sp = _sample_points(p)
        dth = C.on_points(torch.func.jacfwd(C.theta), sp)          # (N, 3)
        gtu = C.on_points(C.gtu_of, sp)                            # (N, 3, 3)
        ex = 2.0 * np.einsum("nij,nj->in", gtu, dth).reshape((3,) + d.shape[1:]) * a
        e = max(np.abs(d[GAM[i]] - ex[i]).max() for i in range(3))
        for i in range(3):
            np.testing.assert_allclose(d[BV[i]], d[GAM[i]], rtol=0, atol=1e-13 * scale)
        assert np.abs(ex).max() > 0.05
        errs[n] = e
    assert errs[32] < 1e-4 and np.log2(errs[16] / errs[32]) > 3.5, errs


def test_theta_shift_lapse_variants():
    """The 1+log source with Khat (lapse_uses_khat) moves by -2 alpha (-2 theta)
    = 4 alpha theta under the shift above; the harmonic lapse (-alpha^2 K)
    does not move."""
    p, pts, u1 = C.patch_state(16)
    th = _field(C.theta, pts, p.shape[1:])
    u2 = u1.copy()
    u2[TH] += th
    u2[KH] -= 2.0 * th
    a, ts = _at(p, u1[ALP]), _at(p, th)
    pk = oracle.Params(lapse_uses_khat=1)
    d = _at(p, oracle.rhs(p, u2, pk, terms=1) - oracle.rhs(p, u1, pk, terms=1))[ALP]
    np.testing.assert_allclose(d, 4.0 * a * ts, rtol=1e-12, atol=1e-15)
    ph = oracle.Params(lapse=1)
    d = _at(p, oracle.rhs(p, u2, ph, terms=1) - oracle.rhs(p, u1, ph, terms=1))[ALP]
    np.testing.assert_allclose(d, 0.0, atol=1e-15)


def _constant_state(p, W, al, gt, Kh, Th, At, Gam, be, B):
    u = np.zeros(p.shape)
    u[0] = W
    for a in range(6):
        u[1 + a] = gt[a]
        u[9 + a] = At[a]
    u[KH], u[TH], u[ALP] = Kh, Th, al
    for i in range(3):
        u[GAM[i]], u[19 + i], u[BV[i]] = Gam[i], be[i], B[i]
    return u


def _sym(c):
    return np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])


def _six(m):
    return np.array([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


@pytest.mark.parametrize("k1,k2", [(0.005, 0.0), (0.4, 0.0), (0.4, 0.3)])
@pytest.mark.parametrize("lapse,khat", [(0, 0), (0, 1), (1, 0)])
def test_constant_data_closed_form(k1, k2, lapse, khat):
    """Spatially constant W, alpha, gt (det 1, off-diagonal), Khat, Theta, At
    (trace-free), Gamt, beta, B: every derivative, the advection and the
    dissipation vanish exactly, and each right-hand side is the algebraic part
    of its equation, evaluated from the physical gamma_ij = gt_ij / W^2 and
    K_ij = (At_ij + gt_ij K / 3) / W^2 with K = Khat + 2 Theta by the ADM
    route (d_t gamma_ij = -2 alpha K_ij, d_t K_ij = alpha (K K_ij - 2 K_ik
    K^k_j), d_t alpha by the slicing) plus the damping terms."""
    p = idd.centred_patch(8, 0.5)
    g = _sym([1.1, 0.05, -0.03, 0.95, 0.02, 1.0])
    g = g / np.linalg.det(g) ** (1.0 / 3.0)
    gtu = np.linalg.inv(g)
    A = _sym([0.03, -0.01, 0.02, 0.015, 0.005, 0.0])
    A[2, 2] -= np.trace(gtu @ A) / gtu[2, 2]  # trace-free w.r.t. gt
    W, al, Kh, Th = 0.9, 0.8, 0.1, 0.02
    Gam, be, B = np.array([0.01, -0.02, 0.015]), np.array([0.1, -0.05, 0.2]), np.array([0.03, 0.01, -0.02])
    u = _constant_state(p, W, al, _six(g), Kh, Th, _six(A), Gam, be, B)
    eta = 0.36
    r = oracle.rhs(p, u, oracle.Params(kappa1=k1, kappa2=k2, eta=eta, lapse=lapse, lapse_uses_khat=khat))
    r = r[:, 3:-3, 3:-3, 3:-3]

    K = Kh + 2.0 * Th
    gam = g / W ** 2
    gamu = np.linalg.inv(gam)
    Kij = (A + g * K / 3.0) / W ** 2
    Kmix = gamu @ Kij                       # K^i_j
    KK = np.trace(Kmix @ Kmix)              # K_ij K^ij
    dgam = -2.0 * al * Kij                  # ADM, constant alpha, any (constant) shift
    dKij = al * (K * Kij - 2.0 * Kij @ Kmix)
    dgamu = -gamu @ dgam @ gamu
    dKtr = np.trace(dgamu @ Kij) + np.trace(gamu @ dKij)
    dW = -W / 6.0 * np.trace(gamu @ dgam)   # W = det(gamma)^(-1/6)
    dg = 2.0 * W * dW * gam + W ** 2 * dgam
    dA = 2.0 * W * dW * (Kij - gam * K / 3.0) + W ** 2 * (dKij - dgam * K / 3.0 - gam * dKtr / 3.0)
    # Khat = K - 2 Theta from the damped Z4 system (flat, constant data):
    # d_t K = alpha ((K - 2 Theta) K - 3 k1 (1 + k2) Theta),
    # d_t Theta = alpha/2 ((K - 2 Theta) K - K_ij K^ij - 2 k1 (2 + k2) Theta)
    z4_dK = al * ((K - 2.0 * Th) * K - 3.0 * k1 * (1.0 + k2) * Th)
    z4_dTh = 0.5 * al * ((K - 2.0 * Th) * K - KK - 2.0 * k1 * (2.0 + k2) * Th)
    dKh = z4_dK - 2.0 * z4_dTh
    # Z4c's Theta equation keeps alpha/2 (K^2 - K_ij K^ij) of the Z4 term and
    # drops its non-principal -alpha Theta K
    dTh = z4_dTh + al * Th * K
    # Gamt: the Z4c damping -2 alpha k1 (Gamt - Gamd), Gamd = 0 here
    dGam = -2.0 * al * k1 * Gam
    dal = -al * al * K if lapse == 1 else -2.0 * al * (Kh if khat else K)
    ex = np.concatenate([[dW], _six(dg), [dKh, dTh], _six(dA), dGam, [dal], 0.75 * B, dGam - eta * B])
    for f in range(25):
        np.testing.assert_allclose(r[f], ex[f], rtol=1e-12, atol=1e-15, err_msg=idd.FIELD_NAMES[f])
