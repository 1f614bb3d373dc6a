"""Continuum reference for the oracle pins, computed by a route that shares
nothing with the oracle: the ADM (3+1) vacuum equations written with the
physical metric, its Christoffel symbols and Ricci tensor by definition, and
exact derivatives from torch autograd (float64, CPU).

For data with Theta = 0 and Gamt^i = -d_j gt^ij (the Gamma constraint
satisfied), the Z4c right-hand side reduces to the ADM time derivatives of the
conformal variables plus constraint additions that the Z4c/BSSN derivation
fixes:
  d_t Khat  = d_t K|ADM - alpha H            (Theta absorbs alpha H / 2)
  d_t Theta = alpha H / 2
  d_t Gamt^i = d_t(-d_j gt^ij)|ADM + 2 alpha gt^ij M_j
with H = R + K^2 - K_ij K^ij and M_j = D_i (K^i_j - delta^i_j K) the vacuum
Hamiltonian and momentum constraints (Sec. 2.3).
"""
from __future__ import annotations

import math

import torch
from torch.func import jacfwd, vmap

torch.set_default_dtype(torch.float64)

EPS = 0.15


def _sym(c):
    """6 components (xx,xy,xz,yy,yz,zz) -> 3x3 symmetric tensor."""
    return torch.stack([torch.stack([c[0], c[1], c[2]]), torch.stack([c[1], c[3], c[4]]),
                        torch.stack([c[2], c[4], c[5]])])


def det3(m):
    """3x3 determinant by cofactors (explicit arithmetic: vmap/jacfwd safe)."""
    return (m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1])
            - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
            + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0]))


def inv3(m):
    """3x3 inverse by the adjugate."""
    c = [[m[(j + 1) % 3, (i + 1) % 3] * m[(j + 2) % 3, (i + 2) % 3]
          - m[(j + 1) % 3, (i + 2) % 3] * m[(j + 2) % 3, (i + 1) % 3] for j in range(3)] for i in range(3)]
    adj = torch.stack([torch.stack(row) for row in c])
    return adj / det3(m)


def _six(m):
    return torch.stack([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


# ------------------------------------------------------------- smooth generic data
PI = math.pi


def gamma(x):
    X, Y, Z = x[0], x[1], x[2]
    c = [1.0 + EPS * torch.sin(PI * X + 0.3) * torch.cos(0.5 * PI * Y),
         0.5 * EPS * torch.sin(PI * (X + Y) + 0.1),
         0.4 * EPS * torch.cos(PI * Z - 0.2) * torch.sin(0.5 * PI * X + 0.4),
         1.0 + EPS * torch.cos(PI * Y - 0.5) * torch.sin(0.7 * PI * Z + 0.2),
         0.3 * EPS * torch.sin(PI * (Y - Z) + 0.7),
         1.0 + EPS * torch.sin(PI * Z + 0.9) * torch.cos(0.6 * PI * X)]
    return _sym(c)


def Kij(x):
    X, Y, Z = x[0], x[1], x[2]
    c = [0.3 * torch.cos(PI * X + 0.2) * torch.sin(0.5 * PI * Z + 0.1),
         0.2 * torch.sin(PI * Y - 0.4),
         0.25 * torch.cos(PI * (X - Z)),
         -0.2 * torch.sin(PI * X + 0.6) * torch.cos(PI * Y),
         0.15 * torch.cos(PI * Y + 0.3),
         0.1 * torch.sin(PI * (X + Z) + 0.5)]
    return _sym(c)


def alpha(x):
    return 0.8 + 0.1 * torch.sin(PI * x[0] + 0.2) * torch.cos(0.5 * PI * x[1] - 0.3) + 0.05 * torch.cos(PI * x[2])


def beta(x):
    X, Y, Z = x[0], x[1], x[2]
    return torch.stack([0.2 * torch.sin(PI * Y + 0.4) + 0.1 * torch.cos(PI * Z),
                        -0.15 * torch.cos(PI * X - 0.2) * torch.sin(0.5 * PI * Z + 0.6),
                        0.1 * torch.sin(PI * (X + Y) - 0.5)])


def Bvec(x):
    X, Y, Z = x[0], x[1], x[2]
    return torch.stack([0.1 * torch.cos(PI * Z + 0.2), 0.05 * torch.sin(PI * X),
                        -0.08 * torch.cos(PI * Y - 0.1)])


# ------------------------------------------------------------- conformal variables

def W_of(x):
    return det3(gamma(x)) ** (-1.0 / 6.0)


def gt_of(x):
    return W_of(x) ** 2 * gamma(x)


def gtu_of(x):
    return inv3(gt_of(x))


def Ktr_of(x):
    return torch.einsum("ij,ij->", inv3(gamma(x)), Kij(x))


def At_of(x):
    return W_of(x) ** 2 * (Kij(x) - gamma(x) * Ktr_of(x) / 3.0)


def Gamt_of(x):
    dgtu = jacfwd(gtu_of)(x)  # [i, j, k] = d_k gt^ij
    return -torch.einsum("ijj->i", dgtu)


def z4c_state(x):
    """All 25 evolved fields at one point."""
    return torch.cat([W_of(x)[None], _six(gt_of(x)), Ktr_of(x)[None], torch.zeros(1), _six(At_of(x)),
                      Gamt_of(x), alpha(x)[None], beta(x), Bvec(x)])


# ------------------------------------------------------------- ADM by definition

def christoffel(x):
    """Gamma^k_ij of the physical metric: [k, i, j]."""
    g = gamma(x)
    gu = inv3(g)
    dg = jacfwd(gamma)(x)  # [i, j, k] = d_k g_ij
    # Gamma_lij = 1/2 (d_i g_lj + d_j g_il - d_l g_ij)
    low = 0.5 * (torch.einsum("lji->lij", dg) + torch.einsum("ilj->lij", dg)
                 - torch.einsum("ijl->lij", dg))
    return torch.einsum("kl,lij->kij", gu, low)


def ricci(x):
    G = christoffel(x)
    dG = jacfwd(christoffel)(x)  # [k, i, j, m] = d_m Gamma^k_ij
    t1 = torch.einsum("kijk->ij", dG)
    t2 = torch.einsum("kikj->ij", dG)
    t3 = torch.einsum("kkl,lij->ij", G, G)
    t4 = torch.einsum("kjl,lik->ij", G, G)
    return t1 - t2 + t3 - t4


def lie_cov(T_fn, x):
    """Lie derivative of a covariant 2-tensor along beta."""
    T = T_fn(x)
    dT = jacfwd(T_fn)(x)  # [i, j, k] = d_k T_ij
    b = beta(x)
    db = jacfwd(beta)(x)  # [k, i] = d_i beta^k
    return (torch.einsum("k,ijk->ij", b, dT) + torch.einsum("kj,ki->ij", T, db)
            + torch.einsum("ik,kj->ij", T, db))


def dt_gamma(x):
    return -2.0 * alpha(x) * Kij(x) + lie_cov(gamma, x)


# ------------------------------------------------------------- perfect fluid

FLUID_EOS = {"K": 100.0, "Gamma": 2.0, "Gamma_th": 1.8}


def fluid(x):
    """Generic smooth primitives (rho, eps, u_i) of a perfect fluid, eps above
    the cold curve of FLUID_EOS (a positive thermal part)."""
    X, Y, Z = x[0], x[1], x[2]
    rho = 3e-3 * (1.0 + 0.3 * torch.sin(PI * X + 0.2) * torch.cos(0.5 * PI * Z) + 0.2 * torch.cos(PI * Y - 0.4))
    K, G = FLUID_EOS["K"], FLUID_EOS["Gamma"]
    eps = K * rho ** (G - 1.0) / (G - 1.0) * (1.3 + 0.2 * torch.sin(PI * (X - Y) + 0.3))
    ul = torch.stack([0.35 * torch.sin(PI * Y + 0.5), -0.3 * torch.cos(PI * (X + Z)),
                      0.3 * torch.sin(PI * Z - 0.3) * torch.cos(0.5 * PI * X) + 0.1])
    return rho, eps, ul


def fluid_pressure(rho, eps):
    """Polytropic cold part plus thermal part, P = K rho^G + (G_th - 1) rho (eps - eps_cold)."""
    K, G, Gt = FLUID_EOS["K"], FLUID_EOS["Gamma"], FLUID_EOS["Gamma_th"]
    ec = K * rho ** (G - 1.0) / (G - 1.0)
    return K * rho ** G + (Gt - 1.0) * rho * (eps - ec)


def tmunu_31(x):
    """rho_ADM = n n T, S_i = -gamma_i^mu n^nu T_{mu nu}, S_ij = gamma gamma T of
    T_{mu nu} = rho h u_mu u_nu + P g_{mu nu}, from the 4-velocity's spatial
    covariant components u_i and n_mu u^mu = -W_L (W_L the Lorentz factor)."""
    rho, eps, ul = fluid(x)
    P = fluid_pressure(rho, eps)
    h = 1.0 + eps + P / rho
    g = gamma(x)
    gu = inv3(g)
    WL = torch.sqrt(1.0 + ul @ gu @ ul)
    E = rho * h * WL ** 2 - P
    S = rho * h * WL * ul
    Sij = rho * h * torch.outer(ul, ul) + P * g
    return E, S, Sij


def dt_K(x, matter=False):
    """d_t K_ij (ADM; with matter the -8 pi alpha (S_ij - gamma_ij (S - rho)/2)
    source)."""
    G = christoffel(x)
    da = jacfwd(alpha)(x)
    dda = jacfwd(jacfwd(alpha))(x)
    DDa = dda - torch.einsum("kij,k->ij", G, da)
    K = Kij(x)
    gu = inv3(gamma(x))
    Kmix = torch.einsum("kl,lj->kj", gu, K)  # K^k_j
    trK = torch.einsum("kk->", Kmix)
    out = (-DDa + alpha(x) * (ricci(x) - 2.0 * torch.einsum("ik,kj->ij", K, Kmix) + trK * K)
           + lie_cov(Kij, x))
    if matter:
        E, _, Sij = tmunu_31(x)
        Str = torch.einsum("ij,ij->", gu, Sij)
        out = out - 8.0 * PI * alpha(x) * (Sij - 0.5 * gamma(x) * (Str - E))
    return out


def constraints_adm(x, matter=False):
    """Hamiltonian H and covariant momentum constraint M_j (with matter:
    -16 pi rho_ADM and -8 pi S_j)."""
    g = gamma(x)
    gu = inv3(g)
    K = Kij(x)
    trK = torch.einsum("ij,ij->", gu, K)
    KK = torch.einsum("ia,jb,ij,ab->", gu, gu, K, K)
    R = torch.einsum("ij,ij->", gu, ricci(x))
    H = R + trK ** 2 - KK
    G = christoffel(x)
    dK = jacfwd(Kij)(x)  # [k, j, i] = d_i K_kj
    # D_i K_kj = d_i K_kj - Gamma^l_ik K_lj - Gamma^l_ij K_kl
    DK = (torch.einsum("kji->ikj", dK) - torch.einsum("lik,lj->ikj", G, K)
          - torch.einsum("lij,kl->ikj", G, K))
    dtrK = jacfwd(Ktr_of)(x)
    M = torch.einsum("ik,ikj->j", gu, DK) - dtrK
    if matter:
        E, Sl, _ = tmunu_31(x)
        H = H - 16.0 * PI * E
        M = M - 8.0 * PI * Sl
    return H, M


def dt_W(x):
    gu = inv3(gamma(x))
    return -W_of(x) / 6.0 * torch.einsum("ij,ij->", gu, dt_gamma(x))


def dt_gt(x):
    return 2.0 * W_of(x) * dt_W(x) * gamma(x) + W_of(x) ** 2 * dt_gamma(x)


def dt_Ktr(x, matter=False):
    gu = inv3(gamma(x))
    dgu = -gu @ dt_gamma(x) @ gu
    return torch.einsum("ij,ij->", dgu, Kij(x)) + torch.einsum("ij,ij->", gu, dt_K(x, matter))


def dt_At(x, matter=False):
    W = W_of(x)
    K = Ktr_of(x)
    return (2.0 * W * dt_W(x) * (Kij(x) - gamma(x) * K / 3.0)
            + W ** 2 * (dt_K(x, matter) - dt_gamma(x) * K / 3.0 - gamma(x) * dt_Ktr(x, matter) / 3.0))


def dt_gtu(x):
    gu = gtu_of(x)
    return -gu @ dt_gt(x) @ gu


def dt_Gamt_kinematic(x):
    d = jacfwd(dt_gtu)(x)  # [i, j, k] = d_k (d_t gt^ij)
    return -torch.einsum("ijj->i", d)


def z4c_rhs_continuum(x, eta=0.36, matter=False):
    """Expected Z4c RHS (no dissipation) for this data, 25 fields (with the
    fluid of tmunu_31 as matter when `matter`)."""
    H, M = constraints_adm(x, matter)
    a = alpha(x)
    b = beta(x)
    gtu = gtu_of(x)
    rW = dt_W(x)
    rgt = _six(dt_gt(x))
    rTh = 0.5 * a * H
    rKh = dt_Ktr(x, matter) - a * H
    rAt = _six(dt_At(x, matter))
    rG = dt_Gamt_kinematic(x) + 2.0 * a * (gtu @ M)
    K = Ktr_of(x)
    ra = -2.0 * a * K + b @ jacfwd(alpha)(x)
    db = jacfwd(beta)(x)
    rb = 0.75 * Bvec(x) + db @ b
    dG = jacfwd(Gamt_of)(x)
    dB = jacfwd(Bvec)(x)
    rB = rG - dG @ b + dB @ b - eta * Bvec(x)
    return torch.cat([rW[None], rgt, rKh[None], rTh[None], rAt, rG, ra[None], rb, rB])


def constraints_continuum(x, matter=False):
    """H and M^i (index raised with the physical metric)."""
    H, M = constraints_adm(x, matter)
    gu = inv3(gamma(x))
    return torch.cat([H[None], gu @ M])


def on_points(fn, pts):
    """Evaluate fn at an (N, 3) float64 array of points, in chunks."""
    import numpy as np
    out = []
    P = torch.as_tensor(pts)
    for s in range(0, P.shape[0], 2048):
        out.append(vmap(fn)(P[s:s + 2048]).detach().numpy())
    return np.concatenate(out, axis=0)


# ------------------------------------------------------------- Theta and Z data

def theta(x):
    """A smooth, generic Theta(x) (O(0.05)) for the damping-term pins."""
    X, Y, Z = x[0], x[1], x[2]
    return 0.05 * torch.sin(PI * X + 0.4) * torch.cos(0.5 * PI * Z - 0.2) + 0.03 * torch.cos(PI * Y + 0.1)


def gam_offset(x):
    """A smooth vector added to the evolved Gamt^i, so that Gamt^i - Gamd^i
    (twice the conformal Z4 vector, gt^ij Z_j) is non-zero."""
    X, Y, Z = x[0], x[1], x[2]
    return torch.stack([0.04 * torch.cos(PI * Y - 0.3), -0.03 * torch.sin(PI * (X + Z) + 0.2),
                        0.05 * torch.cos(PI * X) * torch.sin(0.5 * PI * Y + 0.7)])


_PATCH_CACHE = {}


def patch_state(n):
    """The n^3 patch on [-1/2, 1/2]^3 (ghosts included) with the generic data
    of z4c_state at every cell centre, as a (25, n+6, n+6, n+6) array; cached
    per n for the test session."""
    import numpy as np

    import initial_data as idd

    if n not in _PATCH_CACHE:
        p = idd.Patch(n=(n, n, n), dx=1.0 / n, origin=(-0.5, -0.5, -0.5))
        z, y, xx = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
        pts = np.stack([xx.ravel(), y.ravel(), z.ravel()], axis=1)
        u = np.ascontiguousarray(on_points(z4c_state, pts).T.reshape(p.shape))
        _PATCH_CACHE[n] = (p, pts, u)
    return _PATCH_CACHE[n]


def fluid_prims(x):
    """(rho, eps, u_x, u_y, u_z) at one point, for the grid arrays."""
    rho, eps, ul = fluid(x)
    return torch.cat([rho[None], eps[None], ul])
