"""CPU FP64 oracle of the GR hydrodynamics (matter) sector -- test
infrastructure only (the tests and the benchmark's CPU arm use it; the
product library never does).

Written from the paper's description (Sec. 2.1.2, 2.2) in numpy, plain and
vectorised over the grid, one operation of the method after the other:

* Perfect fluid (Sec. 2.1.2): T^{mu nu} = rho h u^mu u^nu + P g^{mu nu},
  h = 1 + eps + P/rho.  Primitive variables (rho, eps, u_i), u_i the spatial
  covariant components of the four-velocity; Lorentz factor of the Eulerian
  observer w = alpha u^t = sqrt(1 + gamma^{ij} u_i u_j).  Conserved
  variables D = rho w, J_i = rho h w u_i, rho_H = rho h w^2 - P, evolved
  densitised with sqrt(gamma): (D^, J^_i, E^) = sqrt(gamma) (D, J_i, rho_H).
* Hybrid EOS (Sec. 2.1.2): P = P_cold(rho) + (Gamma_th - 1) rho (eps -
  eps_cold(rho)), the cold part a piecewise polytrope P = K_i rho^Gamma_i
  (continuous P and eps, d eps_cold = P_cold / rho^2 d rho).
* Evolution (the 3+1 form of div T = 0 and div(rho u) = 0), with the
  coordinate velocity V^j = alpha gamma^{jk} u_k / w - beta^j:
    d_t D^   + d_j (D^ V^j)                                   = 0
    d_t J^_i + d_j (J^_i V^j + alpha sqrt(gamma) P delta^j_i) =
        sqrt(gamma) (-rho_H d_i alpha + J_k d_i beta^k + alpha/2 S^{jk} d_i gamma_jk)
    d_t E^   + d_j (E^ V^j + sqrt(gamma) P (V^j + beta^j))    =
        sqrt(gamma) (alpha S^{jk} K_jk - J^j d_j alpha)
  with S^{jk} = rho h u^j u^k + P gamma^{jk}, u^j = gamma^{jk} u_k.
* Finite volume (Sec. 2.2): the primitives are reconstructed at the cell
  faces with PPM (Colella & Woodward 1984) whose slopes are limited by the
  steep minmod with b = 3; the face flux is the HLLC flux of special
  relativity (Mignone & Bodo 2005) solved in an orthonormal tetrad in which
  the face is at rest, with the HLLE flux there where the intermediate state
  is unphysical, transformed back to the coordinate frame (an HLLE flux in
  the coordinate frame is kept as an option); the metric at a face is the
  4th-order Lagrange interpolation (-1, 9, 9, -1)/16 of the cell values; the
  metric derivatives of the sources are the 4th-order centred differences
  of the spacetime.
* Primitive recovery (Sec. 2.2): Newton-Raphson on w.  With rho = D/w and
  h = (rho_H + P)/(D w), the hybrid EOS gives P as an explicit function of
  w, P(w) = [P_cold + (G-1)(rho_H/w^2 - (D/w)(1 + eps_cold))] /
  [1 + (G-1)(1 - 1/w^2)], G = Gamma_th, and the root of
  f(w) = w - (rho_H + P) / sqrt((rho_H + P)^2 - S^2), S^2 = gamma^{ij} J_i
  J_j, is the Lorentz factor.
* Atmosphere (Sec. 2.2): a cell below the density floor, or whose recovery
  fails, is reset to rest at the floor density on the cold curve; the floor
  is f_atm rho_max (f_atm = 1e-12) inside r_atm and falls as r^-3 outside.
* Coupling to Z4c: rho_ADM = rho_H, S_i = J_i, S_ij = rho h u_i u_j + P
  gamma_ij enter d_t Khat += 4 pi alpha (S + rho_ADM), d_t Theta -= 8 pi
  alpha rho_ADM, d_t At_ij -= 8 pi alpha W^2 (S_ij - gamma_ij S/3),
  d_t Gamt^i -= 16 pi alpha gt^ij S_j (and B^i through Gamt^i), and the
  constraints H -= 16 pi rho_ADM, M_i -= 8 pi S_i.

Readings where the paper is silent are listed in the design notes: the
tetrad (e1 along the gradient of the face coordinate, e0 the Eulerian
observer projected onto the face), the HLLE fallback also where the contact
speed has no real root or leaves the outer waves, no PPM contact steepening
or flattening, the
repair eps -> eps_cold when the recovered thermal energy is negative,
outflow (zero-gradient) ghost cells on the outer boundary.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

NP = 5  # rho, eps, u_x, u_y, u_z  /  D^, J^_x, J^_y, J^_z, E^
SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
ALP, BETX, W_, GXX, KH, TH, AXX, GAMX, BX = 18, 19, 0, 1, 7, 8, 9, 15, 22


# ------------------------------------------------------------------ EOS

@dataclasses.dataclass
class EOS:
    """Piecewise polytrope cold part + thermal part (Sec. 2.1.2).  Pieces
    i = 0..n-1: P = K_i rho^Gamma_i on [rho_{i}, rho_{i+1}) with rho_0 = 0;
    K_0 given, the other K_i fixed by continuity of P at the boundaries."""
    K0: float
    gammas: Sequence[float]
    rho_bounds: Sequence[float] = ()  # n-1 boundaries, increasing
    gamma_th: float = 1.8

    def __post_init__(self):
        n = len(self.gammas)
        assert len(self.rho_bounds) == n - 1
        self.K = [self.K0]
        self.a = [0.0]
        for i in range(1, n):
            rb, g0, g1 = self.rho_bounds[i - 1], self.gammas[i - 1], self.gammas[i]
            Ki = self.K[i - 1] * rb ** (g0 - g1)
            self.K.append(Ki)
            # eps continuous at rb
            e_prev = self.a[i - 1] + self.K[i - 1] * rb ** (g0 - 1.0) / (g0 - 1.0)
            self.a.append(e_prev - Ki * rb ** (g1 - 1.0) / (g1 - 1.0))

    def _piece(self, rho):
        idx = np.zeros(np.shape(rho), dtype=int)
        for b in self.rho_bounds:
            idx = idx + (np.asarray(rho) >= b)
        return idx

    def cold(self, rho):
        """(P_cold, eps_cold, dP_cold/drho) at rho."""
        rho = np.asarray(rho, dtype=np.float64)
        i = self._piece(rho)
        K = np.asarray(self.K)[i]
        G = np.asarray(self.gammas)[i]
        a = np.asarray(self.a)[i]
        P = K * rho ** G
        eps = a + K * rho ** (G - 1.0) / (G - 1.0)
        dP = G * K * rho ** (G - 1.0)
        return P, eps, dP

    def pressure(self, rho, eps):
        Pc, ec, _ = self.cold(rho)
        return Pc + (self.gamma_th - 1.0) * rho * (eps - ec)

    def cs2(self, rho, eps):
        """Sound speed squared (dP/drho|_eps + P/rho^2 dP/deps|_rho) / h."""
        Pc, ec, dPc = self.cold(rho)
        g = self.gamma_th - 1.0
        P = Pc + g * rho * (eps - ec)
        chi = dPc + g * (eps - ec) - g * Pc / rho  # d eps_cold / d rho = P_cold / rho^2
        kap = g * rho
        h = 1.0 + eps + P / rho
        return (chi + P / rho ** 2 * kap) / h


# ------------------------------------------------------------------ metric

def _sym3(c):
    return np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])


def _inv_sym(g):
    """Inverse of a symmetric 3x3 field (6 components, cofactors / det)."""
    c0 = g[3] * g[5] - g[4] * g[4]
    c1 = g[2] * g[4] - g[1] * g[5]
    c2 = g[1] * g[4] - g[2] * g[3]
    det = g[0] * c0 + g[1] * c1 + g[2] * c2
    inv = np.array([c0, c1, c2, g[0] * g[5] - g[2] * g[2], g[1] * g[2] - g[0] * g[4], g[0] * g[3] - g[1] * g[1]])
    return inv / det, det


def metric(u):
    """3+1 quantities from the Z4c state (25, ...): alpha, beta^i, gamma_ij,
    gamma^ij, sqrt(gamma), K_ij."""
    W = u[W_]
    gt = u[GXX:GXX + 6]
    gtu, detgt = _inv_sym(gt)
    g_ll = gt / W ** 2
    g_uu = gtu * W ** 2
    sqrtg = np.sqrt(detgt) / W ** 3
    K = u[KH] + 2.0 * u[TH]
    K_ll = (u[AXX:AXX + 6] + gt * K / 3.0) / W ** 2
    return {"alpha": u[ALP], "beta": u[BETX:BETX + 3], "g_ll": g_ll, "g_uu": g_uu, "sqrtg": sqrtg,
            "K_ll": K_ll}


def _raise(g_uu, v):
    """v^i = gamma^ij v_j."""
    return np.array([sum(g_uu[SYM[i][j]] * v[j] for j in range(3)) for i in range(3)])


# ------------------------------------------------------------------ prim <-> con

def prim2con(prim, m, eos):
    """Densitised conserved variables (D^, J^_i, E^) and (w, h, P)."""
    rho, eps, ul = prim[0], prim[1], prim[2:5]
    uu = _raise(m["g_uu"], ul)
    w = np.sqrt(1.0 + (ul * uu).sum(axis=0))
    P = eos.pressure(rho, eps)
    h = 1.0 + eps + P / rho
    sg = m["sqrtg"]
    cons = np.empty_like(prim)
    cons[0] = sg * rho * w
    cons[1:4] = sg * rho * h * w * ul
    cons[4] = sg * (rho * h * w * w - P)
    return cons, w, h, P


def _pressure_of_w(w, D, E, eos):
    rho = D / w
    Pc, ec, _ = eos.cold(rho)
    g = eos.gamma_th - 1.0
    return (Pc + g * (E / w ** 2 - (D / w) * (1.0 + ec))) / (1.0 + g * (1.0 - 1.0 / w ** 2))


def _residual(w, D, E, S2, eos):
    P = _pressure_of_w(w, D, E, eos)
    q = (E + P) ** 2 - S2
    return w - (E + P) / np.sqrt(np.maximum(q, 1e-300)), P, q


def con2prim(cons, m, eos, w_guess=None, tol=1e-15, maxit=60):
    """Primitives from densitised conserved variables by Newton-Raphson on
    the Lorentz factor w (numerical derivative; bisection on the bracket
    [1, w_hi] where Newton leaves it), starting from w_guess (default 1).
    Returns (prim, ok): ok false where no physical root exists (atmosphere
    is applied by the caller).  For very hot and dense states on a stiff
    polytrope piece f(w) can have two roots; the iteration returns the one
    it reaches from the guess."""
    sg = m["sqrtg"]
    D, J, E = cons[0] / sg, cons[1:4] / sg, cons[4] / sg
    S2 = (J * _raise(m["g_uu"], J)).sum(axis=0)
    w = np.ones_like(D) if w_guess is None else np.array(w_guess, dtype=np.float64, copy=True)
    # bracket: w >= 1; (rho_H + P) >= sqrt(S2) bounds w from above through E
    lo = np.ones_like(D)
    hi = np.full_like(D, 1e4)
    ok = np.isfinite(D) & (D > 0) & np.isfinite(E) & (E > 0)
    w = np.where(ok, np.clip(w, 1.0, 1e4), 1.0)
    for _ in range(maxit):
        f, _, _ = _residual(w, D, E, S2, eos)
        dw = 1e-7 * w
        f1, _, _ = _residual(w + dw, D, E, S2, eos)
        fp = (f1 - f) / dw
        lo = np.where(f < 0, np.maximum(lo, w), lo)
        hi = np.where(f > 0, np.minimum(hi, w), hi)
        wn = w - f / np.where(fp != 0, fp, 1.0)
        # the bracket is closed: w = 1 (a fluid at rest) is a root
        out = ~((wn >= lo) & (wn <= hi)) | ~np.isfinite(wn)
        wn = np.where(out, 0.5 * (lo + hi), wn)
        done = np.abs(wn - w) <= tol * wn
        w = wn
        if np.all(done | ~ok):
            break
    f, P, q = _residual(w, D, E, S2, eos)
    rho = D / w
    h = (E + P) / (D * w)
    eps = h - 1.0 - P / rho
    ok = ok & np.isfinite(w) & (q > 0) & (rho > 0) & (np.abs(f) <= 1e-10 * w)
    prim = np.empty_like(cons)
    prim[0] = rho
    prim[1] = eps
    prim[2:5] = J / (rho * h * w)
    return prim, ok


def atmosphere_floor(p, rho_max, f_atm=1e-12, r_atm=None):
    """Floor density at every cell of patch p (Sec. 2.2): f_atm rho_max
    within r_atm (default: 8 times the patch's largest extent, the finest
    domain of a one-patch grid), falling as r^-3 outside."""
    if r_atm is None:
        r_atm = 8.0 * max(p.n[d] * p.dx for d in range(3))
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    return f_atm * rho_max * np.where(r <= r_atm, 1.0, (r_atm / np.maximum(r, 1e-300)) ** 3)


def recover(cons, u, eos, floor, w_guess=None):
    """con2prim plus the atmosphere: cells whose density falls below the
    floor or whose recovery fails are reset to rest at the floor density on
    the cold curve; a negative thermal energy is repaired to the cold value.
    The conserved variables of repaired cells are recomputed.  Returns
    (prim, cons, reset mask)."""
    m = metric(u)
    prim, ok = con2prim(cons, m, eos, w_guess)
    _, ec, _ = eos.cold(np.where(ok, prim[0], 1.0))
    low_eps = ok & (prim[1] < ec)
    prim[1] = np.where(low_eps, ec, prim[1])
    reset = ~ok | (prim[0] < floor)
    _, ef, _ = eos.cold(floor)
    prim[0] = np.where(reset, floor, prim[0])
    prim[1] = np.where(reset, ef, prim[1])
    for i in range(3):
        prim[2 + i] = np.where(reset, 0.0, prim[2 + i])
    fix = reset | low_eps
    c2, _, _, _ = prim2con(prim, m, eos)
    cons = np.where(fix[None], c2, cons)
    return prim, cons, reset


# ------------------------------------------------------------------ reconstruction

def _minmod3(a, b, c):
    s = np.sign(a)
    same = (np.sign(b) == s) & (np.sign(c) == s)
    return np.where(same, s * np.minimum(np.minimum(np.abs(a), np.abs(b)), np.abs(c)), 0.0)


def ppm_faces(a, axis, b=3.0):
    """PPM edge values along `axis` (Colella & Woodward 1984) with slopes
    limited by the steep minmod of parameter b (Sec. 2.2).  Returns
    (left, right): left[m] is the state just left of face m+1/2 (cell m's
    right edge), right[m] the state just right of it (cell m+1's left edge),
    valid for m = 2 .. N-4 (other entries NaN)."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0)
    N = a.shape[0]
    nan = np.full_like(a, np.nan)
    # limited slopes at cells 1 .. N-2
    dl = np.full_like(a, np.nan)
    dl[1:-1] = _minmod3(0.5 * (a[2:] - a[:-2]), b * (a[2:] - a[1:-1]), b * (a[1:-1] - a[:-2]))
    # face values a_{m+1/2} for m = 1 .. N-3
    af = nan.copy()
    af[1:-2] = 0.5 * (a[1:-2] + a[2:-1]) - (dl[2:-1] - dl[1:-2]) / 6.0
    # parabola edges of cell i (i = 2 .. N-3): aL = a_{i-1/2}, aR = a_{i+1/2}
    aL, aR = nan.copy(), nan.copy()
    aL[2:-2] = af[1:-3]
    aR[2:-2] = af[2:-2]
    c = a
    ext = (aR - c) * (c - aL) <= 0.0
    aL = np.where(ext, c, aL)
    aR = np.where(ext, c, aR)
    d = aR - aL
    mid = c - 0.5 * (aL + aR)
    over_l = d * mid > d * d / 6.0
    aL = np.where(over_l, 3.0 * c - 2.0 * aR, aL)
    over_r = -d * d / 6.0 > d * mid
    aR = np.where(over_r & ~over_l, 3.0 * c - 2.0 * aL, aR)
    left, right = nan.copy(), nan.copy()
    left[2:N - 3] = aR[2:N - 3]
    right[2:N - 3] = aL[3:N - 2]
    return np.moveaxis(left, 0, axis), np.moveaxis(right, 0, axis)


def face_metric(u, axis):
    """Metric at the faces m+1/2 along axis (m = 1 .. N-3) by the 4th-order
    Lagrange interpolation (-1, 9, 9, -1)/16 of alpha, beta^i, gamma_ij."""
    m = metric(u)
    q = np.concatenate([m["alpha"][None], m["beta"], m["g_ll"]], axis=0)  # (10, ...)
    q = np.moveaxis(q, axis + 1, 1)
    f = np.full_like(q, np.nan)
    f[:, 1:-2] = (-q[:, :-3] + 9.0 * q[:, 1:-2] + 9.0 * q[:, 2:-1] - q[:, 3:]) / 16.0
    f = np.moveaxis(f, 1, axis + 1)
    g_uu, det = _inv_sym(f[4:10])
    return {"alpha": f[0], "beta": f[1:4], "g_ll": f[4:10], "g_uu": g_uu, "sqrtg": np.sqrt(det)}


def _flux(prim, m, eos, d):
    """Conserved variables, physical flux along d and characteristic speeds."""
    cons, w, h, P = prim2con(prim, m, eos)
    rho, eps, ul = prim[0], prim[1], prim[2:5]
    uu = _raise(m["g_uu"], ul)
    al, be, sg = m["alpha"], m["beta"], m["sqrtg"]
    V = al * uu[d] / w - be[d]
    F = cons * V[None]
    F[1 + d] = F[1 + d] + al * sg * P
    F[4] = F[4] + sg * P * (V + be[d])
    # speeds along d (Banyuls et al. 1997): Eulerian v^d = u^d / w
    vd = uu[d] / w
    v2 = 1.0 - 1.0 / w ** 2
    cs2 = eos.cs2(rho, eps)
    gdd = m["g_uu"][SYM[d][d]]
    root = np.sqrt(np.maximum(cs2 * (1.0 - v2) * (gdd * (1.0 - v2 * cs2) - vd * vd * (1.0 - cs2)), 0.0))
    lp = al / (1.0 - v2 * cs2) * (vd * (1.0 - cs2) + root) - be[d]
    lm = al / (1.0 - v2 * cs2) * (vd * (1.0 - cs2) - root) - be[d]
    return cons, F, lp, lm


def hlle_flux(pl, pr, m, eos, d):
    """HLLE flux (Harten-Lax-van Leer-Einfeldt) at faces from the left and
    right primitive states, speeds bounded by 0 on both sides."""
    ul, fl, lpl, lml = _flux(pl, m, eos, d)
    ur, fr, lpr, lmr = _flux(pr, m, eos, d)
    ap = np.maximum(0.0, np.maximum(lpl, lpr))
    am = np.minimum(0.0, np.minimum(lml, lmr))
    den = np.where(ap - am > 0, ap - am, 1.0)
    return (ap[None] * fl - am[None] * fr + (ap * am)[None] * (ur - ul)) / den[None]


# ------------------------------------------------------------------ HLLC in a tetrad frame

def _dot4(m, a, b):
    """g_{mu nu} a^mu b^nu of contravariant 4-vectors (4, ...)."""
    al, be, g = m["alpha"], m["beta"], m["g_ll"]
    bl = np.array([sum(g[SYM[i][j]] * be[j] for j in range(3)) for i in range(3)])
    g00 = -al * al + (bl * be).sum(axis=0)
    out = g00 * a[0] * b[0]
    for i in range(3):
        out = out + bl[i] * (a[0] * b[1 + i] + a[1 + i] * b[0])
        for j in range(3):
            out = out + g[SYM[i][j]] * a[1 + i] * b[1 + j]
    return out


def face_tetrad(m, d):
    """Orthonormal tetrad at faces normal to x^d (Sec. 2.2: the Riemann
    problem is solved in a local Minkowski frame).  e1 is the unit vector
    along the spacetime gradient of x^d, g^{mu d} / sqrt(g^{dd}); e0 is the
    Eulerian observer n projected onto the face's world-sheet x^d = const and
    normalised; e2, e3 are the two coordinate directions along the face made
    orthonormal to e0 (and e2) by Gram-Schmidt.  e0, e2, e3 are tangent to
    the world-sheet, so the face is at rest in this frame.  Returns
    (e (4 vectors, each (4, ...)), sqrt(g^dd))."""
    al, be, gu = m["alpha"], m["beta"], m["g_uu"]
    one, zero = np.ones_like(al), np.zeros_like(al)
    gdd = gu[SYM[d][d]] - be[d] ** 2 / al ** 2
    s1 = np.sqrt(gdd)
    xi = np.array([be[d] / al ** 2] + [gu[SYM[i][d]] - be[i] * be[d] / al ** 2 for i in range(3)])
    e1 = xi / s1
    n = np.array([1.0 / al] + [-be[i] / al for i in range(3)])
    c = -be[d] / al / s1  # n . e1
    e0 = (n - c * e1) / np.sqrt(1.0 + c * c)
    es = []
    for k, a in enumerate(((d + 1) % 3, (d + 2) % 3)):
        v = np.array([zero] + [one if i == a else zero for i in range(3)])
        v = v + _dot4(m, v, e0) * e0
        for q in es:
            v = v - _dot4(m, v, q) * q
        es.append(v / np.sqrt(_dot4(m, v, v)))
    return [e0, e1, es[0], es[1]], s1


def _sr_state(prim, m, eos, e):
    """Special-relativistic state in the tetrad frame: conserved (D, S_1,
    S_2, S_3, E) with E = rho h W^2 - P, the flux along 1, the speeds along
    1 and (v_1, P)."""
    rho, eps, ul = prim[0], prim[1], prim[2:5]
    al, be = m["alpha"], m["beta"]
    uu = _raise(m["g_uu"], ul)
    w = np.sqrt(1.0 + (ul * uu).sum(axis=0))
    u_low = np.array([-al * w + (be * ul).sum(axis=0)] + [ul[i] for i in range(3)])  # u_mu
    comp = [(e[a] * u_low).sum(axis=0) for a in range(4)]
    Wt = -comp[0]
    v = [comp[a] / Wt for a in (1, 2, 3)]
    P = eos.pressure(rho, eps)
    h = 1.0 + eps + P / rho
    U = np.array([rho * Wt, rho * h * Wt * Wt * v[0], rho * h * Wt * Wt * v[1], rho * h * Wt * Wt * v[2],
                  rho * h * Wt * Wt - P])
    F = U * v[0]
    F[1] = F[1] + P
    F[4] = U[1]
    v2 = v[0] ** 2 + v[1] ** 2 + v[2] ** 2
    cs2 = eos.cs2(rho, eps)
    root = np.sqrt(np.maximum(cs2 * (1.0 - v2) * (1.0 - v2 * cs2 - v[0] ** 2 * (1.0 - cs2)), 0.0))
    lp = (v[0] * (1.0 - cs2) + root) / (1.0 - v2 * cs2)
    lm = (v[0] * (1.0 - cs2) - root) / (1.0 - v2 * cs2)
    return U, F, lp, lm, v[0], P


def sr_hllc(UL, FL, lpl, lml, vL, PL, UR, FR, lpr, lmr, vR, PR):
    """HLLC flux of special-relativistic hydrodynamics across an interface at
    rest (Mignone & Bodo 2005), with the HLLE flux where the intermediate
    state is unphysical (Sec. 2.2: a negative intermediate pressure or a
    superluminal contact speed; also no real contact speed or one outside the
    outer waves).  Variables (D, S_1, S_2, S_3, E), E the total energy
    density.  Returns (flux, hllc_used)."""
    lL = np.minimum(lml, lmr)
    lR = np.maximum(lpl, lpr)
    with np.errstate(divide="ignore", invalid="ignore"):  # branches not taken are computed too
        return _sr_hllc(UL, FL, vL, PL, UR, FR, vR, PR, lL, lR)


def _sr_hllc(UL, FL, vL, PL, UR, FR, vR, PR, lL, lR):
    den = lR - lL
    Uh = (lR * UR - lL * UL + FL - FR) / den
    Fh = (lR * FL - lL * FR + lL * lR * (UR - UL)) / den
    # contact speed: F_E^hll l^2 - (E^hll + F_S1^hll) l + S1^hll = 0, the root
    # that stays finite as F_E^hll -> 0
    b = Uh[4] + Fh[1]
    disc = b * b - 4.0 * Fh[4] * Uh[1]
    ls = 2.0 * Uh[1] / (b + np.sqrt(np.maximum(disc, 0.0)))
    ps = Fh[1] - ls * Fh[4]
    ok = (disc >= 0.0) & (ps > 0.0) & (np.abs(ls) < 1.0) & (ls > lL) & (ls < lR)

    def star(U, F, lK, vK, PK):
        r = 1.0 / (lK - ls)
        Us = np.array([U[0] * (lK - vK) * r, (U[1] * (lK - vK) + ps - PK) * r, U[2] * (lK - vK) * r,
                       U[3] * (lK - vK) * r, (U[4] * (lK - vK) + ps * ls - PK * vK) * r])
        return F + lK * (Us - U)

    FsL = star(UL, FL, lL, vL, PL)
    FsR = star(UR, FR, lR, vR, PR)
    hllc = np.where(lL >= 0.0, FL, np.where(ls >= 0.0, FsL, np.where(lR > 0.0, FsR, FR)))
    hlle = np.where(lL >= 0.0, FL, np.where(lR <= 0.0, FR, Fh))
    return np.where(ok, hllc, hlle), ok


def hllc_tetrad_flux(pl, pr, m, eos, d):
    """Face flux of the densitised conserved variables (Sec. 2.2): the
    left and right states in the face tetrad, the special-relativistic HLLC
    flux there, back to the coordinate frame.  With xi = dx^d and
    xi . e_a = 0 for a != 1, the coordinate flux needs only the flux row
    along e1: rho u^d = sqrt(g^dd) F_D and T^d_nu = sqrt(g^dd) [F_E (e0)_nu +
    sum_j F_Sj (e_j)_nu] ((e)_nu lowered), so with sqrt(-g) = alpha
    sqrt(gamma):
        D^   flux: alpha sqrt(gamma) sqrt(g^dd) F_D
        J^_i flux: alpha sqrt(gamma) sqrt(g^dd) [F_E (e0)_i + sum_j F_Sj (e_j)_i]
        E^   flux: alpha sqrt(gamma) (-T^d_nu n^nu)
               = alpha^2 sqrt(gamma) sqrt(g^dd) [F_E e0^t + sum_j F_Sj e_j^t]."""
    e, s1 = face_tetrad(m, d)
    UL, FL, lpl, lml, vL, PL = _sr_state(pl, m, eos, e)
    UR, FR, lpr, lmr, vR, PR = _sr_state(pr, m, eos, e)
    Ft, _ = sr_hllc(UL, FL, lpl, lml, vL, PL, UR, FR, lpr, lmr, vR, PR)
    al, be, g = m["alpha"], m["beta"], m["g_ll"]
    bl = np.array([sum(g[SYM[i][j]] * be[j] for j in range(3)) for i in range(3)])
    pre = al * m["sqrtg"] * s1
    rows = [Ft[4], Ft[1], Ft[2], Ft[3]]  # weights of e0, e1, e2, e3
    out = np.empty_like(Ft)
    out[0] = pre * Ft[0]
    for i in range(3):
        acc = 0.0
        for a in range(4):
            low = bl[i] * e[a][0] + sum(g[SYM[i][j]] * e[a][1 + j] for j in range(3))  # (e_a)_i
            acc = acc + rows[a] * low
        out[1 + i] = pre * acc
    out[4] = pre * al * sum(rows[a] * e[a][0] for a in range(4))
    return out


def face_flux(pl, pr, m, eos, d, solver="hllc"):
    """The face flux of the scheme: "hllc" (Sec. 2.2: HLLC in the face
    tetrad, HLLE there where the intermediate state is unphysical) or
    "hlle" (HLLE in the coordinate frame)."""
    if solver == "hllc":
        return hllc_tetrad_flux(pl, pr, m, eos, d)
    return hlle_flux(pl, pr, m, eos, d)


# ------------------------------------------------------------------ right-hand sides

def _d1(f, axis, h):
    """4th-order centred first derivative (interior cells 2 .. N-3)."""
    f = np.moveaxis(f, axis, 0)
    out = np.full_like(f, np.nan)
    out[2:-2] = (8.0 * (f[3:-1] - f[1:-3]) - (f[4:] - f[:-4])) / (12.0 * h)
    return np.moveaxis(out, 0, axis)


def _act(p):
    g = p.g
    return (slice(g, -g), slice(g, -g), slice(g, -g))


def matter_rhs(p, prim, u, eos, b=3.0, solver="hllc", fluxes_out=None):
    """d_t of the densitised conserved variables at the active cells (ghost
    entries 0): minus the divergence of the face fluxes (`face_flux`) plus
    the geometric sources.  fluxes_out (a list) receives the face fluxes of
    every direction, F[..., m] at face m+1/2 along that direction.  prim (ghosts included) and the Z4c state u give the
    fluid and the metric."""
    out = np.zeros_like(prim)
    a = _act(p)
    h = p.dx
    for d in range(3):
        ax = 2 - d  # array axes are (z, y, x)
        mf = face_metric(u, ax)
        pl = np.empty_like(prim)
        pr = np.empty_like(prim)
        for v in range(NP):
            pl[v], pr[v] = ppm_faces(prim[v], ax)
        F = face_flux(pl, pr, mf, eos, d, solver)  # F[..., m] at face m+1/2
        if fluxes_out is not None:
            fluxes_out.append(F)
        Fm = np.roll(F, 1, axis=ax + 1)    # face m-1/2 at cell m
        div = (F - Fm) / h
        out[(slice(None),) + a] -= div[(slice(None),) + a]
    # geometric sources
    m = metric(u)
    rho, eps, ul = prim[0], prim[1], prim[2:5]
    cons, w, hh, P = prim2con(prim, m, eos)
    uu = _raise(m["g_uu"], ul)
    E = rho * hh * w * w - P
    J = rho * hh * w * ul
    Ju = _raise(m["g_uu"], J)
    Suu = np.array([rho * hh * uu[i] * uu[j] + P * m["g_uu"][SYM[i][j]] for i in range(3) for j in range(i, 3)])
    sg = m["sqrtg"]
    dal = [_d1(m["alpha"], 2 - i, h) for i in range(3)]
    dbe = [[_d1(m["beta"][k], 2 - i, h) for k in range(3)] for i in range(3)]
    dg = [[_d1(m["g_ll"][c], 2 - i, h) for c in range(6)] for i in range(3)]
    pairs = [(i, j) for i in range(3) for j in range(i, 3)]
    for i in range(3):
        sgd = 0.0
        for c, (j, k) in enumerate(pairs):
            sgd = sgd + (1.0 if j == k else 2.0) * Suu[c] * dg[i][c]
        s = -E * dal[i] + sum(J[k] * dbe[i][k] for k in range(3)) + 0.5 * m["alpha"] * sgd
        out[(1 + i,) + a] += (sg * s)[a]
    SK = 0.0
    for c, (j, k) in enumerate(pairs):
        SK = SK + (1.0 if j == k else 2.0) * Suu[c] * m["K_ll"][c]
    sE = m["alpha"] * SK - sum(Ju[j] * dal[j] for j in range(3))
    out[(4,) + a] += (sg * sE)[a]
    return out


def tmunu(prim, u, eos):
    """rho_ADM, S_i, S_ij (6) of the fluid at every cell."""
    m = metric(u)
    rho, eps, ul = prim[0], prim[1], prim[2:5]
    _, w, hh, P = prim2con(prim, m, eos)
    E = rho * hh * w * w - P
    J = rho * hh * w * ul
    Sll = np.array([rho * hh * ul[i] * ul[j] + P * m["g_ll"][SYM[i][j]] for i in range(3) for j in range(i, 3)])
    return E, J, Sll


def z4c_matter_rhs(prim, u, eos, frozen_shift=False):
    """Matter terms of the Z4c right-hand side (25 fields, every cell):
    Khat += 4 pi alpha (S + rho), Theta -= 8 pi alpha rho,
    At_ij -= 8 pi alpha W^2 (S_ij - gamma_ij S / 3), Gamt^i -= 16 pi alpha
    gt^ij S_j, and the same Gamt term in B^i (the Gamma driver carries
    d_t Gamt; not with a frozen shift)."""
    E, J, Sll = tmunu(prim, u, eos)
    m = metric(u)
    al, W = u[ALP], u[W_]
    gtu, _ = _inv_sym(u[GXX:GXX + 6])
    S = sum((1.0 if i == j else 2.0) * m["g_uu"][SYM[i][j]] * Sll[SYM[i][j]] for i in range(3) for j in range(i, 3))
    out = np.zeros_like(u)
    out[KH] = 4.0 * math.pi * al * (S + E)
    out[TH] = -8.0 * math.pi * al * E
    for c in range(6):
        out[AXX + c] = -8.0 * math.pi * al * W ** 2 * (Sll[c] - m["g_ll"][c] * S / 3.0)
    for i in range(3):
        gi = -16.0 * math.pi * al * sum(gtu[SYM[i][j]] * J[j] for j in range(3))
        out[GAMX + i] = gi
        if not frozen_shift:
            out[BX + i] = gi
    return out


def matter_constraint_terms(prim, u, eos):
    """Additions to the vacuum H and M^i of the constraint monitor: -16 pi
    rho_ADM and -8 pi W^2 gt^ij S_j (M with its index raised)."""
    E, J, _ = tmunu(prim, u, eos)
    m = metric(u)
    Ju = _raise(m["g_uu"], J)
    return -16.0 * math.pi * E, -8.0 * math.pi * Ju


def outflow_ghosts(p, prim):
    """Zero-gradient outer boundary: every ghost cell takes the primitives of
    the nearest active cell (faces, edges and corners alike)."""
    g = p.g
    out = prim.copy()
    for ax in (1, 2, 3):
        n = out.shape[ax]
        idx = np.clip(np.arange(n), g, n - g - 1)
        out = np.take(out, idx, axis=ax)
    return out


# ------------------------------------------------------------------ time step

def periodic_ghosts(p, prim):
    """Periodic ghost cells along every axis (for tests on periodic boxes)."""
    g = p.g
    out = prim
    for ax in (1, 2, 3):
        n = out.shape[ax]
        idx = (np.arange(n) - g) % (n - 2 * g) + g
        out = np.take(out, idx, axis=ax)
    return out


def rk4_step_cowling(p, cons, u, dt, eos, floor, b=3.0, bc="outflow", solver="hllc"):
    """One classical RK4 step of the matter on the fixed spacetime u
    (Cowling approximation), primitives recovered after every stage update
    (Sec. 2.2) and outflow (or periodic) ghosts.  Returns (cons, prim) of
    the new level."""
    fill = outflow_ghosts if bc == "outflow" else periodic_ghosts

    def prims(c):
        pr, c2, _ = recover(c, u, eos, floor)
        return fill(p, pr), c2

    a = (slice(None),) + _act(p)
    pr, c0 = prims(cons)
    k = matter_rhs(p, pr, u, eos, b, solver)
    y = c0 + dt / 6.0 * k
    cs = c0 + 0.5 * dt * k
    for s, (cw, bw) in enumerate([(0.5, 1.0 / 3.0), (1.0, 1.0 / 3.0), (None, 1.0 / 6.0)]):
        pr, cs = prims(cs)
        k = matter_rhs(p, pr, u, eos, b, solver)
        if cw is None:
            new = y + bw * dt * k
        else:
            y = y + bw * dt * k
            nxt = c0 + cw * dt * k
            cs = nxt
    new = np.where(np.isfinite(new), new, c0)
    out = c0.copy()
    out[a] = new[a]
    pr, out = prims(out)
    return out, pr


def rk4_step_coupled(p, u, cons, dt, eos, floor, prm, bc="sommerfeld", b=3.0, solver="hllc"):
    """One classical RK4 step of the Z4c spacetime and the matter together
    (method of lines, Sec. 2.2): at every stage the primitives are recovered
    from the stage's conserved variables (atmosphere applied, outflow or
    periodic ghosts), the Z4c stage runs with the matter terms of those
    primitives added to its right-hand side, and the matter stage uses the
    stage's metric.  Spacetime ghosts: bc "sommerfeld" (evolved with the
    stage), "frozen" (held fixed) or "periodic" (filled before every stage
    and after the step).  Returns (u, cons, prim) of the new level (prim
    recovered from it)."""
    import oracle as z4c
    fillm = periodic_ghosts if bc == "periodic" else outflow_ghosts
    a = (slice(None),) + _act(p)
    un = np.array(u, dtype=np.float64, copy=True)
    if bc == "periodic":
        un = z4c.fill_periodic(p, un)
    y = np.zeros_like(un)
    cur = un
    pr, c0, _ = recover(cons, un, eos, floor)
    pr = fillm(p, pr)
    cs = c0
    ym = np.zeros_like(c0)
    cw = [0.5, 0.5, 1.0, None]
    bw = [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]
    for s in range(1, 5):
        if s > 1:
            if bc == "periodic":
                cur = z4c.fill_periodic(p, cur)
            pr, cs, _ = recover(cs, cur, eos, floor)
            pr = fillm(p, pr)
        src = z4c_matter_rhs(pr, cur, eos, frozen_shift=prm.shift == 1)
        out = np.empty_like(un)
        z4c.rk4_stage(p, prm, s, dt, bc == "sommerfeld", cur, un, y, out, src)
        km = matter_rhs(p, pr, cur, eos, b, solver)
        nxt = cs.copy()
        if s == 1:
            ym[a] = c0[a] + bw[0] * dt * km[a]
        elif s < 4:
            ym[a] = ym[a] + bw[s - 1] * dt * km[a]
        if s < 4:
            nxt[a] = c0[a] + cw[s - 1] * dt * km[a]
        else:
            nxt[a] = ym[a] + bw[3] * dt * km[a]
        cur, cs = out, nxt
    if bc == "periodic":
        cur = z4c.fill_periodic(p, cur)
    pr, cs, _ = recover(cs, cur, eos, floor)
    return cur, cs, fillm(p, pr)
