"""Seeded synthetic inputs for the Z4c hot path.

This module only builds inputs: patch geometry, analytic initial data and
counter-based noise.  It holds none of the evolution arithmetic (no
derivative, right-hand side, time step or inter-level operator), so both the
CPU oracle and the CUDA library can be fed from it without sharing any of the
method's code.

Initial data (the paper evolves FUKA data, which is not available; these
analytic families stand in for it):

* Minkowski: W = alpha = 1, gt_ij = delta_ij, every other field 0.
* Brill-Lindquist punctures (time-symmetric, conformally flat): psi = 1 +
  sum_a m_a / (2 |x - x_a|), W = psi^-2, gt_ij = delta_ij, K = At = Gamt = 0,
  precollapsed lapse alpha = psi^-2, beta = B = 0.
* Bowen-York puncture: the Brill-Lindquist conformal factor of one puncture
  with the Bowen-York extrinsic curvature of spin S and momentum P (Bowen &
  York 1980), K_ij = psi^-2 Ahat_ij, Ahat_ij = 3/r^3 (eps_kil S^l n^k n_j +
  eps_kjl S^l n^k n_i) + 3/(2 r^2) (P_i n_j + P_j n_i - (delta_ij - n_i n_j)
  P.n), so At_ij = psi^-6 Ahat_ij; K = 0.  The Hamiltonian constraint is not
  re-solved (psi stays 1 + m/(2r)): an input, not a solution.
* Linearised plane gravitational wave along the unit vector k: in TT gauge
  g_ij = delta_ij + h_+(u) (e1 e1 - e2 e2)_ij + h_x(u) (e1 e2 + e2 e1)_ij,
  u = t - k.x, h_+ = A sin(w u), h_x = B cos(w u), (e1, e2) the theta and phi
  unit vectors of the direction k; K_ij = -d_t g_ij / 2, alpha = 1, beta = 0,
  split into W, gt, Khat = K, At; Gamt = 0 (its exact value is second order
  in the amplitude).
* Gauge wave (Alcubierre et al. 2004 test-bed form): H = 1 - A sin(2 pi (x - t)/d),
  ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2, converted to the W/Z4c variables.
* Noise: uniform in [-a, a] added to every field at every point; the value at
  (field, level-global cell i, j, k) is a SplitMix64 (Steele, Lea & Flood 2014)
  counter hash of the seed and that index, so any implementation can regenerate
  it independently.
* pi symmetrisation (Sec. 3.2): points with x < 0 take the value of their
  partner (-x, -y, z) times the field's parity sign.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

NF = 25
FIELD_NAMES = [
    "W", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "Khat", "Theta",
    "At_xx", "At_xy", "At_xz", "At_yy", "At_yz", "At_zz", "Gamt_x", "Gamt_y", "Gamt_z",
    "alpha", "beta_x", "beta_y", "beta_z", "B_x", "B_y", "B_z",
]
# sign of each field under rotation by pi about z (x -> -x, y -> -y)
PI_PARITY = np.array([
    1, 1, 1, -1, 1, -1, 1, 1, 1, 1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1, -1, 1, -1, -1, 1,
], dtype=np.float64)

# sign of each field under reflection z -> -z (odd number of z indices: -1)
Z_PARITY = np.array([
    1, 1, 1, -1, 1, -1, 1, 1, 1, 1, 1, -1, 1, -1, 1, 1, 1, -1, 1, 1, 1, -1, 1, 1, -1,
], dtype=np.float64)

GHOST = 3


@dataclasses.dataclass
class Patch:
    """A cubic-cell patch: n active cells per axis, ghost width g, spacing dx,
    origin = coordinate of the lower face of active cell 0, refinement level."""
    n: Sequence[int]
    dx: float
    origin: Sequence[float]
    level: int = 0
    g: int = GHOST

    @property
    def shape(self):
        return (NF, self.n[2] + 2 * self.g, self.n[1] + 2 * self.g, self.n[0] + 2 * self.g)

    def axis(self, d: int) -> np.ndarray:
        """Cell-centre coordinates along axis d, ghosts included."""
        idx = np.arange(-self.g, self.n[d] + self.g, dtype=np.float64)
        return self.origin[d] + (idx + 0.5) * self.dx

    def global_index(self, d: int, level_origin: float) -> np.ndarray:
        """Level-global integer cell index along axis d (cells counted from
        level_origin, which must be aligned with this patch's faces)."""
        off = int(round((self.origin[d] - level_origin) / self.dx))
        return np.arange(-self.g, self.n[d] + self.g, dtype=np.int64) + off

    @property
    def active_points(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def centred_patch(n: int, dx: float, centre=(0.0, 0.0, 0.0), level: int = 0) -> Patch:
    return Patch(n=(n, n, n), dx=dx,
                 origin=tuple(c - 0.5 * n * dx for c in centre), level=level)


# ---------------------------------------------------------------- analytic data

def minkowski(p: Patch) -> np.ndarray:
    u = np.zeros(p.shape)
    for f in (0, 1, 4, 6, 18):
        u[f] = 1.0
    return u


def punctures(p: Patch, masses: Sequence[float], positions: Sequence[Sequence[float]]) -> np.ndarray:
    """Brill-Lindquist punctures with precollapsed lapse."""
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    psi = np.ones_like(x)
    for m, c in zip(masses, positions):
        dxp = x - c[0]
        dyp = y - c[1]
        dzp = z - c[2]
        r = np.sqrt(dxp * dxp + dyp * dyp + dzp * dzp)
        psi = psi + m / (2.0 * r)
    W = 1.0 / (psi * psi)
    u = minkowski(p)
    u[0] = W
    u[18] = W
    return u


def bowen_york(p: Patch, mass: float, centre=(0.0, 0.0, 0.0), spin=(0.0, 0.0, 0.0),
               momentum=(0.0, 0.0, 0.0)) -> np.ndarray:
    """One puncture with Bowen-York spin and linear momentum (see module doc)."""
    u = punctures(p, [mass], [centre])
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    xs = [x - centre[0], y - centre[1], z - centre[2]]
    r = np.sqrt(xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2)
    n = [c / r for c in xs]
    S, P = spin, momentum
    # (S x n)_i = eps_ikl S^k n^l, equal to eps_kil S^l n^k
    sxn = [S[1] * n[2] - S[2] * n[1], S[2] * n[0] - S[0] * n[2], S[0] * n[1] - S[1] * n[0]]
    pn = P[0] * n[0] + P[1] * n[1] + P[2] * n[2]
    psi6 = u[0] ** 3  # W^3 = psi^-6
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for a, (i, j) in enumerate(sym):
        ahat = 3.0 / r ** 3 * (sxn[i] * n[j] + sxn[j] * n[i])
        ahat = ahat + 1.5 / r ** 2 * (P[i] * n[j] + P[j] * n[i] - ((1.0 if i == j else 0.0) - n[i] * n[j]) * pn)
        u[9 + a] = psi6 * ahat
    return u


def plane_wave_basis(theta: float, phi: float):
    """Direction k and the polarisation vectors e1 (theta), e2 (phi)."""
    st, ct, sp, cp = math.sin(theta), math.cos(theta), math.sin(phi), math.cos(phi)
    return (np.array([st * cp, st * sp, ct]), np.array([ct * cp, ct * sp, -st]), np.array([-sp, cp, 0.0]))


def plane_wave(p: Patch, amp_plus: float, amp_cross: float, omega: float, theta: float, phi: float,
               t: float = 0.0) -> np.ndarray:
    """Linearised plane wave along the direction (theta, phi) (module doc)."""
    k, e1, e2 = plane_wave_basis(theta, phi)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    uu = t - (k[0] * x + k[1] * y + k[2] * z)
    hp, hx = amp_plus * np.sin(omega * uu), amp_cross * np.cos(omega * uu)
    dhp, dhx = amp_plus * omega * np.cos(omega * uu), -amp_cross * omega * np.sin(omega * uu)
    g = np.zeros((3, 3) + x.shape)
    kk = np.zeros((3, 3) + x.shape)
    for i in range(3):
        for j in range(3):
            ep = e1[i] * e1[j] - e2[i] * e2[j]
            ex = e1[i] * e2[j] + e2[i] * e1[j]
            g[i, j] = (1.0 if i == j else 0.0) + hp * ep + hx * ex
            kk[i, j] = -0.5 * (dhp * ep + dhx * ex)
    gm = np.moveaxis(g, (0, 1), (-2, -1))
    W = np.linalg.det(gm) ** (-1.0 / 6.0)
    gu = np.moveaxis(np.linalg.inv(gm), (-2, -1), (0, 1))
    K = np.einsum("ij...,ij...->...", gu, kk)
    u = minkowski(p)
    u[0] = W
    u[7] = K
    for a, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        u[1 + a] = W * W * g[i, j]
        u[9 + a] = W * W * (kk[i, j] - g[i, j] * K / 3.0)
    return u


def gauge_wave(p: Patch, amp: float, d: float = 1.0, t: float = 0.0) -> np.ndarray:
    """Gauge wave along x in W/Z4c variables (harmonic slicing, zero shift)."""
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    ph = 2.0 * math.pi * (x - t) / d
    H = 1.0 - amp * np.sin(ph)
    dH = -amp * np.cos(ph) * 2.0 * math.pi / d
    Kxx = -(math.pi * amp / d) * np.cos(ph) / np.sqrt(H)
    K = Kxx / H
    W = H ** (-1.0 / 6.0)
    u = np.zeros(p.shape)
    u[0] = W
    u[1] = H ** (2.0 / 3.0)
    u[4] = H ** (-1.0 / 3.0)
    u[6] = H ** (-1.0 / 3.0)
    u[7] = K
    u[9] = 2.0 / 3.0 * W * W * Kxx
    u[12] = -1.0 / 3.0 * W * W * K
    u[14] = -1.0 / 3.0 * W * W * K
    u[15] = 2.0 / 3.0 * H ** (-5.0 / 3.0) * dH
    u[18] = np.sqrt(H)
    return u


# ---------------------------------------------------------------- noise

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to state x (state advanced by the
    golden gamma first), elementwise on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN) & _M64
        z = ((z ^ (z >> np.uint64(30))) * _C1) & _M64
        z = ((z ^ (z >> np.uint64(27))) * _C2) & _M64
        return z ^ (z >> np.uint64(31))


def noise_value(seed: int, f: int, i, j, k) -> np.ndarray:
    """Counter-based uniform noise in [-1, 1): h = sm(sm(sm(sm(seed + f) ^ i) ^ j) ^ k),
    value = 2 * (h >> 11) * 2^-53 - 1, with i, j, k taken as two's-complement uint64."""
    s = _splitmix64(np.uint64(seed) + np.uint64(f))
    h = _splitmix64(s ^ np.asarray(i, dtype=np.int64).astype(np.uint64))
    h = _splitmix64(h ^ np.asarray(j, dtype=np.int64).astype(np.uint64))
    h = _splitmix64(h ^ np.asarray(k, dtype=np.int64).astype(np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def add_noise(p: Patch, u: np.ndarray, amp: float, seed: int, level_origin=None) -> np.ndarray:
    """u + amp * noise at every point (ghosts included) and every field."""
    if amp == 0.0:
        return u
    lo = level_origin if level_origin is not None else p.origin
    gi = p.global_index(0, lo[0])
    gj = p.global_index(1, lo[1])
    gk = p.global_index(2, lo[2])
    K, J, I = np.meshgrid(gk, gj, gi, indexing="ij")
    out = u.copy()
    for f in range(NF):
        out[f] = u[f] + amp * noise_value(seed, f, I, J, K)
    return out


def symmetrise_pi(p: Patch, u: np.ndarray) -> np.ndarray:
    """Replace every point with x < 0 by the parity-signed value of its partner
    (-x, -y, z).  The patch must be centred on x = y = 0."""
    nx = u.shape[3]
    out = u.copy()
    half = nx // 2
    mirrored = u[:, :, ::-1, ::-1] * PI_PARITY[:, None, None, None]
    out[:, :, :, :half] = mirrored[:, :, :, :half]
    return out


# ---------------------------------------------------------------- workloads

PUNCTURE_SEED = 20260743
STABILITY_SEED = 20260744


def single_puncture_patch(n: int = 32, half_width: float = 8.0) -> Patch:
    """Uniform patch [-half_width, half_width]^3 with n^3 cells."""
    return centred_patch(n, 2.0 * half_width / n)


def single_puncture_data(p: Patch, mass: float = 1.0, noise: float = 1e-10,
                         seed: int = PUNCTURE_SEED, pi_symmetric: bool = False) -> np.ndarray:
    u = punctures(p, [mass], [(0.0, 0.0, 0.0)])
    u = add_noise(p, u, noise, seed)
    if pi_symmetric:
        u = symmetrise_pi(p, u)
    return u


@dataclasses.dataclass
class Hierarchy:
    """Static box-in-box hierarchy: patches per level, coarsest spacing dx0."""
    dx0: float
    levels: List[List[Patch]]
    masses: Sequence[float]
    positions: Sequence[Sequence[float]]

    @property
    def patches(self) -> List[Patch]:
        return [p for lv in self.levels for p in lv]

    def zone_updates_per_coarse_step(self) -> int:
        return sum((2 ** l) * sum(p.active_points for p in lv) for l, lv in enumerate(self.levels))


def box_in_box(n_fixed: int, n_moving: int, n_levels: int, n_fixed_levels: int, dx0: float,
               masses, positions) -> Hierarchy:
    """Fixed levels: one n_fixed^3 patch centred on the origin.  Moving levels:
    one n_moving^3 patch centred on each puncture."""
    levels = []
    for l in range(n_levels):
        dx = dx0 / (2 ** l)
        if l < n_fixed_levels:
            levels.append([centred_patch(n_fixed, dx, level=l)])
        else:
            levels.append([centred_patch(n_moving, dx, centre=c, level=l) for c in positions])
    return Hierarchy(dx0=dx0, levels=levels, masses=masses, positions=positions)


def binary_7_level() -> Hierarchy:
    """7 levels: L0-L4 one 96^3 patch (dx 4 .. 1/4), L5-L6 two 64^3 patches
    around equal-mass Brill-Lindquist punctures at (+-5, 0, 0)."""
    return box_in_box(96, 64, 7, 5, 4.0, [0.5, 0.5], [(5.0, 0.0, 0.0), (-5.0, 0.0, 0.0)])


def binary_10_level() -> Hierarchy:
    """10 levels: L0-L5 one 192^3 patch (dx 4 .. 1/8), L6-L9 two 160^3 patches
    around unequal-mass punctures m=0.6 at (+4,0,0) and m=0.4 at (-6,0,0)."""
    return box_in_box(192, 160, 10, 6, 4.0, [0.6, 0.4], [(4.0, 0.0, 0.0), (-6.0, 0.0, 0.0)])


def small_binary(n_fixed: int = 24, n_moving: int = 16, n_levels: int = 4, n_fixed_levels: int = 2,
                 dx0: float = 1.0, sep: float = 2.0) -> Hierarchy:
    """Scaled-down version of the 7-level hierarchy for oracle parity runs."""
    return box_in_box(n_fixed, n_moving, n_levels, n_fixed_levels, dx0, [0.5, 0.5],
                      [(sep, 0.0, 0.0), (-sep, 0.0, 0.0)])


def moving_binary_3_level() -> Hierarchy:
    """3 levels with room for the moving patches: L0 32^3 (dx 1), L1 two
    24^3 (dx 1/2) and L2 two 16^3 (dx 1/4) centred on Brill-Lindquist
    punctures m = 0.5 at (+-3, 0, 0)."""
    pos = [(3.0, 0.0, 0.0), (-3.0, 0.0, 0.0)]
    levels = [[centred_patch(32, 1.0, level=0)],
              [centred_patch(24, 0.5, centre=c, level=1) for c in pos],
              [centred_patch(16, 0.25, centre=c, level=2) for c in pos]]
    return Hierarchy(dx0=1.0, levels=levels, masses=[0.5, 0.5], positions=pos)


def nesting_ok(h: Hierarchy, margin: int = 4) -> bool:
    """Every patch of level l > 0 lies inside a patch of level l-1, aligned with
    its cell faces, with at least `margin` parent cells around it."""
    for l in range(1, len(h.levels)):
        for c in h.levels[l]:
            ok_any = False
            for p in h.levels[l - 1]:
                ok = True
                for d in range(3):
                    t = (c.origin[d] - p.origin[d]) / p.dx
                    if abs(t - round(t)) > 1e-9 or c.n[d] % 2:
                        ok = False
                    off = int(round(t))
                    if off - margin < 0 or off + c.n[d] // 2 + margin - 1 > p.n[d] - 1:
                        ok = False
                ok_any |= ok
            if not ok_any:
                return False
    return True


def level_origin(h: Hierarchy, level: int):
    """Origin used for level-global cell indices: the coarsest patch's origin
    refined to this level (every patch of the level is aligned with it)."""
    return tuple(h.levels[0][0].origin)


def symmetrise_z(p: Patch, u: np.ndarray) -> np.ndarray:
    """Make data on a patch centred on z = 0 exactly symmetric under z -> -z:
    every point with z < 0 takes Z_PARITY times its mirror's value."""
    nz = u.shape[1]
    assert nz % 2 == 0 and abs(p.origin[2] + 0.5 * p.n[2] * p.dx) < 1e-12 * p.dx
    v = np.array(u, copy=True)
    v[:, : nz // 2] = Z_PARITY[:, None, None, None] * v[:, nz // 2:][:, ::-1]
    return v


def upper_half(p: Patch) -> Patch:
    """The z >= 0 half of a patch centred on z = 0."""
    assert p.n[2] % 2 == 0 and abs(p.origin[2] + 0.5 * p.n[2] * p.dx) < 1e-12 * p.dx
    return Patch(n=(p.n[0], p.n[1], p.n[2] // 2), dx=p.dx, origin=(p.origin[0], p.origin[1], 0.0),
                 level=p.level, g=p.g)


def upper_half_array(p: Patch, u: np.ndarray) -> np.ndarray:
    """The array of upper_half(p) (ghosts included) cut from the full one."""
    nz = p.n[2]
    return np.ascontiguousarray(u[:, nz // 2: nz // 2 + nz // 2 + 2 * p.g])


def upper_half_hierarchy(h: Hierarchy) -> Hierarchy:
    return Hierarchy(dx0=h.dx0, levels=[[upper_half(p) for p in lv] for lv in h.levels],
                     masses=h.masses, positions=h.positions)


def hierarchy_data(h: Hierarchy, noise: float = 0.0, seed: int = PUNCTURE_SEED) -> List[np.ndarray]:
    out = []
    for lv in h.levels:
        for p in lv:
            u = punctures(p, h.masses, h.positions)
            out.append(add_noise(p, u, noise, seed, level_origin(h, p.level)))
    return out
