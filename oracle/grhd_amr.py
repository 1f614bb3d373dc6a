"""CPU FP64 oracle of the matter sector on the Berger-Oliger hierarchy --
test infrastructure only (the tests use it; the product library never
does).

Written from the paper's description of its mesh refinement for the fluid
(Sec. 2.2.1), with the hierarchy, the time levels and the spacetime's
prolongation, restriction and time interpolation of the oracle's
BOHierarchy (oracle/__init__.py):

* Prolongation of the fluid onto a child's ghost cells (the 3-cell
  refinement boundary): the conserved rest-mass density, densitised
  D^ = sqrt(gamma) rho w, by a conservative fifth-order WENO interpolation
  (Jiang & Shu smoothness indicators on the three 3-cell stencils, applied
  along x, then y, then z; the two children of a parent cell average to
  it); eps and u_i by the spacetime's 6th-order Lagrange interpolation.
  Where the WENO value is unphysical (D^ <= 0) it falls back to the parent
  cell's value, and eps there, or wherever its interpolant is <= 0, falls
  back to trilinear interpolation.  The child's rho is D^ / (sqrt(gamma) w)
  with the child's own metric.
* Time: every parent time level is prolonged, and the child's ghost values
  at a stage time are the time interpolant of those (quadratic through three
  levels, linear through two, as for the spacetime).
* Restriction: a parent cell under a child's active cells takes the volume
  average of its 8 children's densitised conserved variables.
* Reflux: for a parent cell outside a child that shares a face with the
  child's active region, the parent step's flux through that face (the
  RK4-weighted sum of its stage fluxes) is replaced by the children's: the
  RK4-weighted fluxes through the 4 fine faces, averaged over the face and
  over the child's two steps.  With periodic or no-flux outer boundaries the
  total rest mass (sum of D^ dV over the cells not covered by a finer level)
  is then conserved to rounding.
* Equatorial reflection symmetry (Sec. 2.2.2: only z >= 0 evolved): the
  fluid's z < 0 ghost layers of a patch on z = 0 mirror the layers above,
  rho, eps, u_x, u_y, D^, J^_x, J^_y, E^ even and u_z, J^_z odd in z, after
  every other ghost treatment; a child on z = 0 is prolonged from its
  parent extended below z = 0 by the same mirror image (the values the
  full domain holds there), and its own z < 0 ghosts are then reflected.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

import oracle as z4c
from oracle import grhd

GAMMA = (3.0 / 16.0, 5.0 / 8.0, 3.0 / 16.0)  # linear weights: the 5-cell quartic's left-half average
RK_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


# ------------------------------------------------------------------ 1D operators on cell averages

def weno5_children(q, axis):
    """Averages over the two halves of every parent cell along `axis` from
    the parent cell averages q.  For parent cell I with neighbours
    a..e = q_{I-2} .. q_{I+2} the left-half averages of the three quadratic
    interpolants are (-a + 4b + 5c)/8, (b + 8c - d)/8, (11c - 4d + e)/8;
    their combination with weights (3/16, 5/8, 3/16) is the left-half
    average of the 5-cell quartic.  The nonlinear weights are
    gamma_k / (eps + beta_k)^2, normalised, with the Jiang-Shu indicators
    beta_k and eps = 1e-6 times the mean square of a..e.  The right half is
    2c - left (the two halves average to the parent).  Output: 2N cells
    along axis (children 2I, 2I+1 of parent I), NaN for the parent cells
    without two neighbours on each side."""
    q = np.moveaxis(np.asarray(q, dtype=np.float64), axis, 0)
    N = q.shape[0]
    out = np.full((2 * N,) + q.shape[1:], np.nan)
    a, b, c, d, e = q[0:N - 4], q[1:N - 3], q[2:N - 2], q[3:N - 1], q[4:N]
    L = [(-a + 4.0 * b + 5.0 * c) / 8.0, (b + 8.0 * c - d) / 8.0, (11.0 * c - 4.0 * d + e) / 8.0]
    B = [13.0 / 12.0 * (a - 2.0 * b + c) ** 2 + 0.25 * (a - 4.0 * b + 3.0 * c) ** 2,
         13.0 / 12.0 * (b - 2.0 * c + d) ** 2 + 0.25 * (b - d) ** 2,
         13.0 / 12.0 * (c - 2.0 * d + e) ** 2 + 0.25 * (3.0 * c - 4.0 * d + e) ** 2]
    eps = 1e-6 * (a * a + b * b + c * c + d * d + e * e) / 5.0 + 1e-300
    al = [GAMMA[k] / (eps + B[k]) ** 2 for k in range(3)]
    s = al[0] + al[1] + al[2]
    left = (al[0] * L[0] + al[1] * L[1] + al[2] * L[2]) / s
    out[4:2 * N - 4:2] = left
    out[5:2 * N - 3:2] = 2.0 * c - left
    return np.moveaxis(out, 0, axis)


def linear_children(q, axis):
    """Linear interpolation at the two child centres (-1/4 and +1/4 of a
    parent cell): 3/4 of the cell plus 1/4 of the neighbour on that side."""
    q = np.moveaxis(np.asarray(q, dtype=np.float64), axis, 0)
    N = q.shape[0]
    out = np.full((2 * N,) + q.shape[1:], np.nan)
    out[2:2 * N - 2:2] = 0.75 * q[1:N - 1] + 0.25 * q[0:N - 2]
    out[3:2 * N - 1:2] = 0.75 * q[1:N - 1] + 0.25 * q[2:N]
    return np.moveaxis(out, 0, axis)


# 6-point Lagrange weights of the child centres at +1/4 (nodes -2..3) and
# -1/4 (nodes -3..2) of a parent cell (the spacetime's prolongation)
LAG_P = np.array([77.0, -693.0, 6930.0, 2310.0, -495.0, 63.0]) / 8192.0
LAG_M = LAG_P[::-1]


def lagrange_children(q, axis):
    """Values at the two child centres of every parent cell along `axis`
    by 6th-order Lagrange interpolation of the parent values q (exact for
    quintics); NaN for parent cells without three neighbours on each side."""
    q = np.moveaxis(np.asarray(q, dtype=np.float64), axis, 0)
    N = q.shape[0]
    out = np.full((2 * N,) + q.shape[1:], np.nan)
    left = sum(LAG_M[m] * q[m:N - 6 + m] for m in range(6))       # nodes I-3 .. I+2, I = 3 .. N-4
    right = sum(LAG_P[m] * q[1 + m:N - 5 + m] for m in range(6))  # nodes I-2 .. I+3
    out[6:2 * N - 6:2] = left[:N - 6]
    out[7:2 * N - 5:2] = right[:N - 6]
    return np.moveaxis(out, 0, axis)


# ------------------------------------------------------------------ equatorial symmetry

PRIM_Z_PARITY = np.array([1.0, 1.0, 1.0, 1.0, -1.0])  # rho, eps, u_x, u_y, u_z
CONS_Z_PARITY = np.array([1.0, 1.0, 1.0, -1.0, 1.0])  # D^, J^_x, J^_y, J^_z, E^


def fill_zreflect_fluid(p, arr, parity):
    """z -> -z mirror of the z < 0 ghost layers of a patch whose lower face
    is z = 0: layer k (k < g, at z = (k - g + 1/2) dx) takes parity times
    layer 2g - 1 - k (at -z)."""
    if not z4c.touches_equator(p):
        raise ValueError("the patch's lower z face is not z = 0")
    g = p.g
    out = np.array(arr, dtype=np.float64, copy=True)
    for k in range(g):
        out[:, k] = parity[:, None, None] * arr[:, 2 * g - 1 - k]
    return out


def mirror_extend(p, arr, parity, rows):
    """A patch on z = 0 and its array extended by `rows` layers below its
    z < 0 ghosts, each the mirror image (layer -m takes parity times layer
    2g - 1 + m): the patch that describes the extended array has its origin
    `rows` cells lower and `rows` more active cells along z."""
    if not z4c.touches_equator(p):
        raise ValueError("the patch's lower z face is not z = 0")
    g = p.g
    below = [parity[:, None, None] * arr[:, 2 * g - 1 + m] for m in range(rows, 0, -1)]
    ext = np.concatenate([np.stack(below, axis=1), arr], axis=1)
    q = dataclasses.replace(p, n=(p.n[0], p.n[1], p.n[2] + rows),
                            origin=(p.origin[0], p.origin[1], p.origin[2] - rows * p.dx))
    return q, ext


# ------------------------------------------------------------------ geometry of a child in its parent

def child_offset(parent, child):
    return [int(round((child.origin[d] - parent.origin[d]) / parent.dx)) for d in range(3)]


def _parent_box(parent, child, arr, margin):
    """Parent array block covering the child's array (ghosts included) plus
    `margin` parent cells on each side; arr is (..., z, y, x) with ghosts."""
    off = child_offset(parent, child)
    g = parent.g
    sl = []
    for d in (2, 1, 0):
        lo = off[d] - 2 - margin + g        # parent cell of child cell -3 is off - 2
        hi = off[d] + child.n[d] // 2 + 1 + margin + g
        if lo < 0 or hi >= arr.shape[-1 - d]:
            raise ValueError("child too close to its parent's edge for the fluid's prolongation")
        sl.append(slice(lo, hi + 1))
    return arr[(Ellipsis,) + tuple(sl)]


def _child_cells(box_children, child, margin):
    """Crop the child-resolution block (children of parent cells off-2-margin
    .. off+n/2+1+margin) to the child's array: child cells -3 .. n+2."""
    k = 2 * margin + 1  # child cell -4 - 2 margin is first; -3 is one later
    sl = tuple(slice(k, k + child.n[d] + 2 * child.g) for d in (2, 1, 0))
    return box_children[(Ellipsis,) + sl]


def weno5_prolong(parent, child, q):
    """The child's array (ghosts included) of a parent cell-average field q
    (parent array with ghosts) by the conservative WENO5, x then y then z."""
    box = _parent_box(parent, child, q, 2)
    for ax in (-1, -2, -3):
        box = weno5_children(box, ax)
    return _child_cells(box, child, 2)


def linear_prolong(parent, child, q):
    box = _parent_box(parent, child, q, 1)
    for ax in (-1, -2, -3):
        box = linear_children(box, ax)
    return _child_cells(box, child, 1)


def parent_cell_values(parent, child, q):
    """The value of the parent cell containing each child cell."""
    box = _parent_box(parent, child, q, 0)
    for ax in (-1, -2, -3):
        box = np.repeat(box, 2, axis=ax)
    return _child_cells(box, child, 0)


def lagrange_prolong(parent, child, fields):
    """6th-order Lagrange prolongation of a few fields onto the child's ghost
    cells (the spacetime's operator, oracle.prolong_ghosts)."""
    nf = len(fields)
    up = np.zeros((z4c.NF,) + fields[0].shape)
    up[:nf] = fields
    uc = np.zeros((z4c.NF,) + tuple(child.n[d] + 2 * child.g for d in (2, 1, 0)))
    uc = z4c.prolong_ghosts(parent, up, child, uc)
    return uc[:nf]


def lagrange_prolong_cells(parent, child, q):
    """The child's whole array of a parent field q by the tensor-product
    6th-order Lagrange interpolation (x, then y, then z)."""
    box = _parent_box(parent, child, q, 3)
    for ax in (-1, -2, -3):
        box = lagrange_children(box, ax)
    return _child_cells(box, child, 3)


def ghost_mask(child):
    g = child.g
    m = np.ones(tuple(child.n[d] + 2 * g for d in (2, 1, 0)), dtype=bool)
    m[g:-g, g:-g, g:-g] = False
    return m


def prolong_fluid(parent, cons_p, prim_p, child, ghosts_only=True):
    """Child ghost values (D^, eps, u_x, u_y, u_z) from one parent time
    level (densitised conserved variables and primitives, arrays with
    ghosts); entries outside the ghost shell are NaN (ghosts_only=False:
    every cell of the child's array)."""
    D = weno5_prolong(parent, child, cons_p[0])
    bad = ~(D > 0.0)
    D = np.where(bad, parent_cell_values(parent, child, cons_p[0]), D)
    if ghosts_only:
        lag = lagrange_prolong(parent, child, [prim_p[1], prim_p[2], prim_p[3], prim_p[4]])
    else:
        lag = [lagrange_prolong_cells(parent, child, prim_p[f]) for f in (1, 2, 3, 4)]
    eps_lin = linear_prolong(parent, child, prim_p[1])
    eps = np.where(bad | ~(lag[0] > 0.0), eps_lin, lag[0])
    out = np.array([D, eps, lag[1], lag[2], lag[3]])
    if ghosts_only:
        out[:, ~ghost_mask(child)] = np.nan
    return out


def ghost_primitives(vals, child, u, eos):
    """Primitives (rho, eps, u_i) at the child's ghost cells from the
    time-interpolated (D^, eps, u_i) and the child's metric u."""
    m = grhd.metric(u)
    ul = vals[2:5]
    uu = grhd._raise(m["g_uu"], ul)
    w = np.sqrt(1.0 + (ul * uu).sum(axis=0))
    rho = vals[0] / (m["sqrtg"] * w)
    return np.array([rho, vals[1], ul[0], ul[1], ul[2]])


# ------------------------------------------------------------------ restriction and reflux

def restrict_fluid(parent, cons_p, child, cons_c):
    """Parent cells under the child's active cells <- mean of their 8
    children (densitised conserved variables)."""
    off = child_offset(parent, child)
    g, gc = parent.g, child.g
    out = np.array(cons_p, copy=True)
    c = cons_c[:, gc:-gc, gc:-gc, gc:-gc]
    avg = 0.125 * (c[:, 0::2, 0::2, 0::2] + c[:, 0::2, 0::2, 1::2] + c[:, 0::2, 1::2, 0::2] +
                   c[:, 0::2, 1::2, 1::2] + c[:, 1::2, 0::2, 0::2] + c[:, 1::2, 0::2, 1::2] +
                   c[:, 1::2, 1::2, 0::2] + c[:, 1::2, 1::2, 1::2])
    nz, ny, nx = child.n[2] // 2, child.n[1] // 2, child.n[0] // 2
    out[:, off[2] + g:off[2] + g + nz, off[1] + g:off[1] + g + ny, off[0] + g:off[0] + g + nx] = avg
    return out


def reflux(parent, cons_p, fbar_p, child, fbar_c, dt_p):
    """Correct the parent cells outside the child next to its boundary:
    the parent's RK4-weighted face fluxes (fbar_p[d][..., m] at face m+1/2
    of array index m along axis d) through the child's boundary faces are
    replaced by the child's, fbar_c averaged over the 4 fine faces (fbar_c
    already averaged over the child's two steps)."""
    off = child_offset(parent, child)
    g, gc = parent.g, child.g
    out = np.array(cons_p, copy=True)
    h = parent.dx
    for d in range(3):
        ax = 3 - d  # array axis of direction d (fields, z, y, x)
        t = [e for e in range(3) if e != d]
        for side in (0, 1):
            # parent face array index along d and the parent cell outside
            if side == 0:
                mp, cell = off[d] - 1 + g, off[d] - 1 + g
                mc = gc - 1
            else:
                mp, cell = off[d] + child.n[d] // 2 - 1 + g, off[d] + child.n[d] // 2 + g
                mc = child.n[d] - 1 + gc
            fp = np.take(fbar_p[d], mp, axis=ax)   # (5, ..) over the two tangential axes
            fc = np.take(fbar_c[d], mc, axis=ax)
            # tangential ranges (array order: the remaining axes are z/y/x minus d)
            sl_p, sl_c = [], []
            for e in sorted(t, reverse=True):  # array order: higher direction first
                sl_p.append(slice(off[e] + g, off[e] + g + child.n[e] // 2))
                sl_c.append(slice(gc, gc + child.n[e]))
            fp = fp[(slice(None),) + tuple(sl_p)]
            fc = fc[(slice(None),) + tuple(sl_c)]
            fine = 0.25 * (fc[:, 0::2, 0::2] + fc[:, 0::2, 1::2] + fc[:, 1::2, 0::2] + fc[:, 1::2, 1::2])
            corr = (dt_p / h) * (fine - fp) * (-1.0 if side == 0 else 1.0)
            idx = [slice(None)] * 4
            idx[ax] = cell
            te = sorted(t, reverse=True)
            for k, e in enumerate(te):
                idx[3 - e] = sl_p[k]
            out[tuple(idx)] = out[tuple(idx)] + corr
    return out


def rest_mass(hierarchy_patches, cons, levels_children):
    """Sum of D^ dV over the cells not covered by a finer level's active
    cells (the composite grid)."""
    total = 0.0
    for pid, p in enumerate(hierarchy_patches):
        g = p.g
        D = np.array(cons[pid][0, g:-g, g:-g, g:-g], copy=True)
        for cid in levels_children[pid]:
            c = hierarchy_patches[cid]
            off = child_offset(p, c)
            D[off[2]:off[2] + c.n[2] // 2, off[1]:off[1] + c.n[1] // 2, off[0]:off[0] + c.n[0] // 2] = 0.0
        total += D.sum() * p.dx ** 3
    return total


# ------------------------------------------------------------------ moving patches (Sec. 2.2.1)

def density_maximum(p, prim):
    """(rho_max, x, y, z): the largest rest-mass density over the patch's
    active cells and that cell's centre (the first in z, y, x order where
    several are equal).  A neutron star is located there."""
    g = p.g
    rho = prim[0, g:-g, g:-g, g:-g]
    k, j, i = np.unravel_index(int(np.argmax(rho)), rho.shape)
    return (float(rho[k, j, i]), p.origin[0] + (i + 0.5) * p.dx, p.origin[1] + (j + 0.5) * p.dx,
            p.origin[2] + (k + 0.5) * p.dx)


def move_fluid(parent, cons_p, prim_p, old, cons_o, prim_o, new, u_new, eos):
    """The fluid of a patch shifted from geometry `old` to `new` (Sec.
    2.2.1): cells active in both keep their conserved variables and
    primitives; every other cell (ghosts included) takes the parent's
    prolongation (D^ conservative WENO5, eps and u_i 6th-order Lagrange,
    with the fallbacks), rho = D^ / (sqrt(gamma) w) with the new metric, and
    the conserved variables of those primitives."""
    vals = prolong_fluid(parent, cons_p, prim_p, new, ghosts_only=False)
    prim = ghost_primitives(vals, new, u_new, eos)
    cons, _, _, _ = grhd.prim2con(prim, grhd.metric(u_new), eos)
    g = new.g
    sh = [int(round((new.origin[d] - old.origin[d]) / new.dx)) for d in range(3)]
    dst, src = [slice(None)], [slice(None)]
    for d in (2, 1, 0):  # new active cell i is old active cell i + sh
        lo, hi = max(0, -sh[d]), min(new.n[d], old.n[d] - sh[d])
        if lo >= hi:
            return cons, prim
        dst.append(slice(g + lo, g + hi))
        src.append(slice(g + lo + sh[d], g + hi + sh[d]))
    cons[tuple(dst)] = cons_o[tuple(src)]
    prim[tuple(dst)] = prim_o[tuple(src)]
    return cons, prim


# ------------------------------------------------------------------ the coupled hierarchy

class MatterHierarchy(z4c.BOHierarchy):
    """The spacetime hierarchy of BOHierarchy with a perfect fluid evolved on
    every level in the same RK4 stages (Sec. 2.2, 2.2.1): per stage and level,
    the primitives recovered from the stage's conserved variables (the
    atmosphere applied), their ghosts filled (level 0: periodic or outflow;
    finer levels: from the parent, above), the Z4c stage with the fluid's
    terms, the fluid's stage with the stage's metric.  After a level's two
    child steps: the spacetime as in BOHierarchy, then the fluid's
    restriction and reflux and the parent's primitives recovered again.
    Patches of one level must not overlap.  With zsym only z >= 0 is
    evolved: spacetime and fluid ghosts below z = 0 by reflection."""

    def __init__(self, hierarchy, states, prims, eos, floors, prm, courant=0.25, bc0=z4c.BC_PERIODIC,
                 solver="hllc", reflux=True, zsym=False):
        super().__init__(hierarchy, states, prm, courant=courant, bc0=bc0, zsym=zsym)
        self.eos, self.floors, self.solver, self.do_reflux = eos, floors, solver, reflux
        self.mbc = "periodic" if bc0 == z4c.BC_PERIODIC else "outflow"
        self.ctl = []  # time levels of (cons, prim) per patch, oldest first
        for pid, (u, pr) in enumerate(zip(states, prims)):
            cons, _, _, _ = grhd.prim2con(pr, grhd.metric(u), eos)
            prn, cons, _ = grhd.recover(cons, u, eos, floors[pid])
            prn = self._fill_level0(pid, prn) if self.patches[pid].level == 0 else prn
            self.ctl.append([self._reflect_fluid(pid, cons, prn)])
        self.fstep = [None] * len(self.patches)  # the last step's RK4-weighted face fluxes
        self.favg = [None] * len(self.patches)   # a child's, averaged over its two steps
        self.children = [[c for c in range(len(self.patches)) if self.parent[c] == pid]
                         for pid in range(len(self.patches))]
        self.follow_star = [-1] * len(self.patches)  # star each patch follows

    def _reflect_fluid(self, pid, cons, prim):
        """(cons, prim) with the z < 0 ghosts mirrored (zsym, patches on z = 0)."""
        if not (self.zsym and z4c.touches_equator(self.patches[pid])):
            return cons, prim
        p = self.patches[pid]
        return fill_zreflect_fluid(p, cons, CONS_Z_PARITY), fill_zreflect_fluid(p, prim, PRIM_Z_PARITY)

    def _fill_level0(self, pid, prim):
        fill = grhd.periodic_ghosts if self.mbc == "periodic" else grhd.outflow_ghosts
        return fill(self.patches[pid], prim)

    def _fluid_ghosts(self, pid, prim, u, frac):
        """Child ghost primitives at fraction frac of the parent's last step."""
        ppid = self.parent[pid]
        levels = self.ctl[ppid]
        w = z4c.time_weights(len(levels), frac)
        src = levels[-3:] if len(levels) >= 3 else [levels[-2], levels[-1]]
        ws = w if len(levels) >= 3 else w[1:]
        vals = None
        on_equator = self.zsym and z4c.touches_equator(self.patches[pid])
        for wi, (cp, pp) in zip(ws, src):
            par = self.patches[ppid]
            if on_equator:  # the stencils reach below z = 0: the parent's mirror image
                _, cp = mirror_extend(par, cp, CONS_Z_PARITY, 2)
                par, pp = mirror_extend(par, pp, PRIM_Z_PARITY, 2)
            v = prolong_fluid(par, cp, pp, self.patches[pid])
            vals = wi * v if vals is None else vals + wi * v
        gp = ghost_primitives(vals, self.patches[pid], u, self.eos)
        mask = ghost_mask(self.patches[pid])
        out = np.array(prim, copy=True)
        out[:, mask] = gp[:, mask]
        return out

    def _prims(self, pid, cons, u, frac):
        pr, cons, _ = grhd.recover(cons, u, self.eos, self.floors[pid])
        if self.patches[pid].level == 0:
            pr = self._fill_level0(pid, pr)
        else:
            pr = self._fluid_ghosts(pid, pr, u, frac)
        cons, pr = self._reflect_fluid(pid, cons, pr)
        return pr, cons

    def _rk4_level(self, l, frac0, dfrac):
        ids = self.level_ids[l]
        dt = self.dt(l)
        un = [self.tl[pid][-1] for pid in ids]
        y = [np.zeros_like(a) for a in un]
        cur = [a.copy() for a in un]
        c0 = [self.ctl[pid][-1][0] for pid in ids]
        cs = [c.copy() for c in c0]
        ym = [np.zeros_like(c) for c in c0]
        fb = [[0.0, 0.0, 0.0] for _ in ids]
        stage_frac = [0.0, 0.5, 0.5, 1.0]
        cw = [0.5, 0.5, 1.0, None]
        evolve_ghosts = (l == 0 and self.bc0 == z4c.BC_SOMMERFELD)
        for s in range(1, 5):
            if l == 0 and self.bc0 == z4c.BC_PERIODIC:
                cur = [z4c.fill_periodic(self.patches[pid], c) for pid, c in zip(ids, cur)]
            if l > 0:
                for a, pid in enumerate(ids):
                    cur[a] = self._fill_child_ghosts(pid, cur[a], frac0 + stage_frac[s - 1] * dfrac)
            cur = self._reflect(ids, cur)
            if s == 1:
                un = [c.copy() for c in cur]
            out = [np.empty_like(a) for a in un]
            for a, pid in enumerate(ids):
                p = self.patches[pid]
                pr, cs[a] = self._prims(pid, cs[a], cur[a], frac0 + stage_frac[s - 1] * dfrac)
                if s == 1:
                    c0[a] = cs[a]
                src = grhd.z4c_matter_rhs(pr, cur[a], self.eos, frozen_shift=self.prm.shift == 1)
                z4c.rk4_stage(p, self.prm, s, dt, evolve_ghosts, cur[a], un[a], y[a], out[a], src)
                fl = []
                km = grhd.matter_rhs(p, pr, cur[a], self.eos, solver=self.solver, fluxes_out=fl)
                for d in range(3):
                    fb[a][d] = fb[a][d] + RK_B[s - 1] * fl[d]
                act = (slice(None),) + grhd._act(p)
                nxt = cs[a].copy()
                if s == 1:
                    ym[a][act] = c0[a][act] + RK_B[0] * dt * km[act]
                elif s < 4:
                    ym[a][act] = ym[a][act] + RK_B[s - 1] * dt * km[act]
                if s < 4:
                    nxt[act] = c0[a][act] + cw[s - 1] * dt * km[act]
                else:
                    nxt[act] = ym[a][act] + RK_B[3] * dt * km[act]
                cs[a] = nxt
            cur = out
        cur = self._reflect(ids, cur)  # the children's prolongation reads these ghosts
        for a, pid in enumerate(ids):
            if l == 0 and self.bc0 == z4c.BC_PERIODIC:
                cur[a] = z4c.fill_periodic(self.patches[pid], cur[a])
            self.tl[pid].append(cur[a])
            if len(self.tl[pid]) > 3:
                self.tl[pid].pop(0)
            pr, cn = self._prims(pid, cs[a], cur[a], frac0 + dfrac)
            self.ctl[pid].append((cn, pr))
            if len(self.ctl[pid]) > 3:
                self.ctl[pid].pop(0)
            # RK4-weighted face fluxes of this step; a child's two steps averaged
            self.fstep[pid] = fb[a]
            if l > 0:
                self.favg[pid] = fb[a] if frac0 == 0.0 else [0.5 * (self.favg[pid][d] + fb[a][d]) for d in range(3)]
        self.nsteps[l] += 1

    def level_step(self, l=0, frac0=0.0, dfrac=1.0):
        self._rk4_level(l, frac0, dfrac)
        if l + 1 < len(self.h.levels):
            self.level_step(l + 1, 0.0, 0.5)
            self.level_step(l + 1, 0.5, 0.5)
            kids = self.level_ids[l + 1]
            for pid in kids:
                self.tl[pid][-1] = self._fill_child_ghosts(pid, self.tl[pid][-1], 1.0)
            for pid, c in zip(kids, self._reflect(kids, [self.tl[pid][-1] for pid in kids])):
                self.tl[pid][-1] = c
            for pid in kids:
                ppid = self.parent[pid]
                self.tl[ppid][-1] = z4c.restrict(self.patches[ppid], self.tl[ppid][-1],
                                                 self.patches[pid], self.tl[pid][-1])
            ids = self.level_ids[l]  # restricted cells next to z = 0 have mirrors among the ghosts
            for pid, c in zip(ids, self._reflect(ids, [self.tl[pid][-1] for pid in ids])):
                self.tl[pid][-1] = c
            # the fluid: restriction, reflux, the parent's primitives again
            for pid in kids:
                ppid = self.parent[pid]
                cp, _ = self.ctl[ppid][-1]
                cp = restrict_fluid(self.patches[ppid], cp, self.patches[pid], self.ctl[pid][-1][0])
                if self.do_reflux:
                    cp = reflux(self.patches[ppid], cp, self.fstep[ppid], self.patches[pid], self.favg[pid],
                                self.dt(l))
                self.ctl[ppid][-1] = (cp, None)
            for ppid in self.level_ids[l]:
                cp, pr = self.ctl[ppid][-1]
                if pr is None:
                    pr, cp = self._prims(ppid, cp, self.tl[ppid][-1], frac0 + dfrac)
                    self.ctl[ppid][-1] = (cp, pr)

    def track_stars(self, follow_star):
        """follow_star[pid] = the star patch pid follows (-1: none).  A star
        is located by the maximum of the rest-mass density on the finest
        patch that follows it (Sec. 2.2.1); regrid() moves its followers."""
        if len(follow_star) != len(self.patches):
            raise ValueError("one entry per patch")
        for pid, s in enumerate(follow_star):
            if s >= 0 and (self.patches[pid].level == 0 or self.follow[pid] >= 0):
                raise ValueError("patch %d cannot follow a star" % pid)
        self.follow_star = [int(v) for v in follow_star]

    def star_positions(self):
        out = {}
        for s in sorted({v for v in self.follow_star if v >= 0}):
            pid = max((q for q, v in enumerate(self.follow_star) if v == s),
                      key=lambda q: (self.patches[q].level, -q))
            out[s] = density_maximum(self.patches[pid], self.prim(pid))[1:]
        return out

    def _targets(self):
        t = super()._targets()
        stars = self.star_positions()
        for pid, s in enumerate(self.follow_star):
            if s >= 0:
                t[pid] = stars[s]
        return t

    def _apply_move(self, pid, shift):
        """The spacetime's move, then the fluid's (move_fluid); the moved
        level's fluid history and, as the parent's cached prolongations of
        its older time levels would need their primitives, the parent
        level's whole history (spacetime and fluid) restart at the current
        time level."""
        old = self.patches[pid]
        oc, op = self.ctl[pid][-1]
        super()._apply_move(pid, shift)
        un = self.tl[pid][-1]
        new = self.patches[pid]
        ppid = self.parent[pid]
        par = self.patches[ppid]
        cp, pp = self.ctl[ppid][-1]
        if self.zsym and z4c.touches_equator(new):
            _, cp = mirror_extend(par, cp, CONS_Z_PARITY, 2)
            par, pp = mirror_extend(par, pp, PRIM_Z_PARITY, 2)
        cons, prim = move_fluid(par, cp, pp, old, oc, op, new, un, self.eos)
        for q in self.level_ids[new.level]:
            self.ctl[q] = [self.ctl[q][-1]]
        self.ctl[pid] = [self._reflect_fluid(pid, cons, prim)]
        for q in self.level_ids[new.level - 1]:
            self.tl[q] = [self.tl[q][-1]]
            self.ctl[q] = [self.ctl[q][-1]]
        return un

    def cons(self, pid):
        return self.ctl[pid][-1][0]

    def prim(self, pid):
        return self.ctl[pid][-1][1]

    def rest_mass(self):
        return rest_mass(self.patches, [self.cons(pid) for pid in range(len(self.patches))], self.children)
