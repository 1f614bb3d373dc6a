"""CPU FP64 oracle of the Z4c hot path -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline arm
may import this package; the product library never does.  The arithmetic is in
``z4c_oracle.c`` (plain C, compiled with -O2 -ffp-contract=off -fno-fast-math,
OpenMP over z-planes); this file loads it and adds the Berger-Oliger driver
(Sec. 2.2.1), which only sequences the C operators.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_z4c.so")
_lock = threading.Lock()
_lib = None

NF = 25


_COUNT_PATH = os.path.join(_BUILD, "flop_count")


def build_flop_count(force: bool = False) -> str:
    """Compile the counting-scalar build of the oracle (flop_count.cpp: the
    oracle's C source with a scalar type that counts its operations)."""
    srcs = [os.path.join(_HERE, f) for f in ("flop_count.cpp", "z4c_oracle.c", "z4c_oracle.h")]
    if not force and os.path.exists(_COUNT_PATH) and os.path.getmtime(_COUNT_PATH) >= max(map(os.path.getmtime, srcs)):
        return _COUNT_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _COUNT_PATH + ".tmp%d" % os.getpid()
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-I" + _HERE, "-o", tmp,
                    srcs[0]], check=True)
    os.replace(tmp, _COUNT_PATH)
    return _COUNT_PATH


def flop_counts(p, u: np.ndarray):
    """FP64 operations per active point of the oracle's evaluation of patch
    array u (centred patch of spacing p.dx): the right-hand side, its
    sources / advection / dissipation parts and one 5-pass RK4 stage; and
    the right-hand side the counting build computed (the oracle's to the bit)."""
    import json
    import tempfile
    exe = build_flop_count()
    with tempfile.TemporaryDirectory() as d:
        fi, fo = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        np.ascontiguousarray(u, dtype=np.float64).tofile(fi)
        r = subprocess.run([exe, str(p.n[0]), str(p.n[1]), str(p.n[2]), repr(float(p.dx)), fi, fo],
                           capture_output=True, text=True, check=True)
        rhs = np.fromfile(fo).reshape(u.shape)
    return json.loads(r.stdout), rhs


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU involved)."""
    src = os.path.join(_HERE, "z4c_oracle.c")
    hdr = os.path.join(_HERE, "z4c_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _OrcPatch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("g", ctypes.c_int), ("dx", ctypes.c_double),
                ("origin", ctypes.c_double * 3)]


class _OrcParams(ctypes.Structure):
    _fields_ = [("kappa1", ctypes.c_double), ("kappa2", ctypes.c_double), ("eta", ctypes.c_double),
                ("sigma_ko", ctypes.c_double), ("w_floor", ctypes.c_double),
                ("lapse", ctypes.c_int), ("shift", ctypes.c_int), ("lapse_uses_khat", ctypes.c_int)]


BC_SOMMERFELD, BC_PERIODIC, BC_FROZEN = 0, 1, 2
BC_ZREFLECT = 8  # or-ed into bc: equatorial reflection symmetry at z = 0 (Sec. 2.2.2)


@dataclasses.dataclass
class Params:
    """Run parameters; defaults are the paper's (Sec. 2.2 and Sec. 3)."""
    kappa1: float = 0.005
    kappa2: float = 0.0
    eta: float = 0.36
    sigma_ko: float = 0.5
    w_floor: float = 1e-10
    lapse: int = 0          # 0: 1+log, 1: harmonic
    shift: int = 0          # 0: Gamma driver, 1: frozen
    lapse_uses_khat: int = 0

    def c(self) -> _OrcParams:
        return _OrcParams(self.kappa1, self.kappa2, self.eta, self.sigma_ko, self.w_floor,
                          self.lapse, self.shift, self.lapse_uses_khat)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            L.orc_z4c_rhs.argtypes = [P(_OrcPatch), P(_OrcParams), dp, dp]
            L.orc_z4c_rhs_terms.argtypes = [P(_OrcPatch), P(_OrcParams), dp, dp, ctypes.c_int]
            L.orc_sommerfeld_rhs.argtypes = [P(_OrcPatch), dp, dp]
            L.orc_fill_periodic.argtypes = [P(_OrcPatch), dp]
            L.orc_fill_zreflect.argtypes = [P(_OrcPatch), dp]
            L.orc_fill_zreflect.restype = ctypes.c_int
            L.orc_prolong_ghosts_ex.argtypes = [P(_OrcPatch), dp, P(_OrcPatch), dp, ctypes.c_int]
            L.orc_enforce.argtypes = [P(_OrcPatch), ctypes.c_double, ctypes.c_int, dp]
            L.orc_rk4_step.argtypes = [P(_OrcPatch), P(_OrcParams), ctypes.c_int, ctypes.c_double, dp]
            L.orc_rk4_stage.argtypes = [P(_OrcPatch), P(_OrcParams), ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, dp, dp, dp, dp]
            L.orc_rk4_stage_src.argtypes = [P(_OrcPatch), P(_OrcParams), ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, dp, dp, dp, dp, dp]
            L.orc_constraints.argtypes = [P(_OrcPatch), dp, ctypes.c_double, dp, dp]
            L.orc_pi_symmetry.argtypes = [P(_OrcPatch), dp, ctypes.c_int]
            L.orc_pi_symmetry.restype = ctypes.c_double
            L.orc_prolong_ghosts.argtypes = [P(_OrcPatch), dp, P(_OrcPatch), dp]
            L.orc_restrict.argtypes = [P(_OrcPatch), dp, P(_OrcPatch), dp]
            L.orc_exchange.argtypes = [P(_OrcPatch), dp, P(_OrcPatch), dp]
            L.orc_exchange.restype = ctypes.c_long
            L.orc_lagrange_weights.argtypes = [ctypes.c_int, P(ctypes.c_int), ctypes.c_double, dp]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_adm_integrals.argtypes = [P(_OrcPatch), dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
            L.orc_adm_integrals.restype = ctypes.c_int
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
            L.orc_move_patch.argtypes = [P(_OrcPatch), dp, P(_OrcPatch), dp, P(_OrcPatch), dp, ctypes.c_int]
            L.orc_move_patch.restype = ctypes.c_int
            L.orc_interp_point.argtypes = [P(_OrcPatch), dp, ctypes.c_int, dp, dp]
            L.orc_interp_point.restype = ctypes.c_int
            L.orc_psi4_point.argtypes = [P(_OrcPatch), dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.orc_psi4_point.restype = ctypes.c_int
            L.orc_psi4_modes.argtypes = [P(_OrcPatch), dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, dp]
            L.orc_psi4_modes.restype = ctypes.c_int
            L.orc_swsh.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.orc_stencils.argtypes = [P(_OrcPatch), dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, dp, dp]
            _lib = L
    return _lib


def _cp(p) -> _OrcPatch:
    return _OrcPatch((ctypes.c_int * 3)(*[int(v) for v in p.n]), int(p.g), float(p.dx),
                     (ctypes.c_double * 3)(*[float(v) for v in p.origin]))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (for timing on a core count)."""
    lib().orc_set_num_threads(int(n))


def rhs(p, u: np.ndarray, prm: Params = Params(), terms: int = 7) -> np.ndarray:
    """Z4c right-hand side at active points (ghost entries 0).
    terms: bit0 sources, bit1 advection, bit2 Kreiss-Oliger."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().orc_z4c_rhs_terms(ctypes.byref(_cp(p)), ctypes.byref(prm.c()), _ptr(u), _ptr(out), terms)
    return out


def sommerfeld_rhs(p, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    lib().orc_sommerfeld_rhs(ctypes.byref(_cp(p)), _ptr(u), _ptr(out))
    return out


def fill_periodic(p, u: np.ndarray) -> np.ndarray:
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    lib().orc_fill_periodic(ctypes.byref(_cp(p)), _ptr(u))
    return u


def fill_zreflect(p, u: np.ndarray) -> np.ndarray:
    """Equatorial reflection (Sec. 2.2.2): the z < 0 ghost layers mirror z > 0
    with the sign of each field's z parity.  The patch's lower z face must be
    z = 0."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    if lib().orc_fill_zreflect(ctypes.byref(_cp(p)), _ptr(u)) != 0:
        raise ValueError("patch does not start at z = 0")
    return u


def touches_equator(p) -> bool:
    return abs(p.origin[2]) <= 1e-12 * p.dx


def enforce(p, u: np.ndarray, w_floor: float = 1e-10, all_points: bool = False) -> np.ndarray:
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    lib().orc_enforce(ctypes.byref(_cp(p)), w_floor, int(all_points), _ptr(u))
    return u


def rk4_step(p, u: np.ndarray, dt: float, prm: Params = Params(), bc: int = BC_SOMMERFELD) -> np.ndarray:
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    lib().orc_rk4_step(ctypes.byref(_cp(p)), ctypes.byref(prm.c()), bc, dt, _ptr(u))
    return u


def rk4_stage(p, prm: Params, s: int, dt: float, evolve_ghosts: bool, us, un, y, out, src=None):
    """RK4 stage s of the Z4c state; src (a patch array or None) is added to
    the right-hand side at the active points (the matter terms)."""
    if src is None:
        lib().orc_rk4_stage(ctypes.byref(_cp(p)), ctypes.byref(prm.c()), s, dt, int(evolve_ghosts),
                            _ptr(us), _ptr(un), _ptr(y), _ptr(out))
    else:
        src = np.ascontiguousarray(src, dtype=np.float64)
        lib().orc_rk4_stage_src(ctypes.byref(_cp(p)), ctypes.byref(prm.c()), s, dt, int(evolve_ghosts),
                                _ptr(us), _ptr(un), _ptr(y), _ptr(out), _ptr(src))


def constraints(p, u: np.ndarray, w_excise: float = 0.0):
    """Returns (c[4, ...] pointwise H, M^x, M^y, M^z; norms[4])."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.empty((4,) + u.shape[1:])
    norms = np.empty(4)
    lib().orc_constraints(ctypes.byref(_cp(p)), _ptr(u), w_excise, _ptr(c), _ptr(norms))
    return c, norms


def pi_symmetry(p, u: np.ndarray, include_ghosts: bool = True) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_pi_symmetry(ctypes.byref(_cp(p)), _ptr(u), int(include_ghosts))


def prolong_ghosts(parent, up: np.ndarray, child, uc: np.ndarray, skip_zlower: bool = False) -> np.ndarray:
    """Ghosts of the child from the parent (skip_zlower: not the z < 0
    layers, which the equatorial reflection fills)."""
    up = np.ascontiguousarray(up, dtype=np.float64)
    uc = np.array(uc, dtype=np.float64, order="C", copy=True)
    rc = lib().orc_prolong_ghosts_ex(ctypes.byref(_cp(parent)), _ptr(up), ctypes.byref(_cp(child)), _ptr(uc),
                                     int(skip_zlower))
    if rc != 0:
        raise ValueError("prolongation stencil leaves the parent patch or patches misaligned")
    return uc


def restrict(parent, up: np.ndarray, child, uc: np.ndarray) -> np.ndarray:
    up = np.array(up, dtype=np.float64, order="C", copy=True)
    uc = np.ascontiguousarray(uc, dtype=np.float64)
    rc = lib().orc_restrict(ctypes.byref(_cp(parent)), _ptr(up), ctypes.byref(_cp(child)), _ptr(uc))
    if rc != 0:
        raise ValueError("child not aligned with / not inside the parent")
    return up


def exchange(a, ua: np.ndarray, b, ub: np.ndarray) -> int:
    """In-place same-level exchange between two patches; returns points touched."""
    n = lib().orc_exchange(ctypes.byref(_cp(a)), _ptr(ua), ctypes.byref(_cp(b)), _ptr(ub))
    if n < 0:
        raise ValueError("patches not aligned")
    return int(n)


def stencils(p, u: np.ndarray, field: int, i: int, j: int, k: int, b=(1.0, 1.0, 1.0)) -> np.ndarray:
    """The RHS's finite-difference operators at one point (array indices incl.
    ghosts): [D_x, D_y, D_z, D_xx, D_yy, D_zz, D_xD_y, D_xD_z, D_yD_z,
    upwind D_x, D_y, D_z for shift b, 6th differences x, y, z]."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty(15)
    lib().orc_stencils(ctypes.byref(_cp(p)), _ptr(u), field, i, j, k, _ptr(bb), _ptr(out))
    return out


def adm_integrals(p, u: np.ndarray, centre, radius: float, ntheta: int = 24, nphi: int = 48):
    """(M_ADM, J_z, P_x, P_y, P_z) on the coordinate sphere of the given
    radius (Sec. 2.3, Sec. 3.2)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    out = np.empty(5)
    rc = lib().orc_adm_integrals(ctypes.byref(_cp(p)), _ptr(u), _ptr(c), float(radius), int(ntheta), int(nphi),
                                 _ptr(out))
    if rc != 0:
        raise ValueError("sphere leaves the patch (interpolation needs 2 cells more)")
    return tuple(float(v) for v in out)


def move_patch(parent, up: np.ndarray, old, uo: np.ndarray, new, skip_zlower: bool = False) -> np.ndarray:
    """Data of a patch shifted from geometry `old` to `new` (Sec. 2.2.1)."""
    up = np.ascontiguousarray(up, dtype=np.float64)
    uo = np.ascontiguousarray(uo, dtype=np.float64)
    un = np.zeros(new.shape)
    rc = lib().orc_move_patch(ctypes.byref(_cp(parent)), _ptr(up), ctypes.byref(_cp(old)), _ptr(uo),
                              ctypes.byref(_cp(new)), _ptr(un), int(skip_zlower))
    if rc != 0:
        raise ValueError("shifted patch misaligned or its prolongation leaves the parent")
    return un


def interp_point(p, u: np.ndarray, f: int, x) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(1)
    if lib().orc_interp_point(ctypes.byref(_cp(p)), _ptr(u), int(f), _ptr(xx), _ptr(out)) != 0:
        raise ValueError("interpolation stencil leaves the active cells")
    return float(out[0])


def psi4_point(p, u: np.ndarray, centre, r: float, theta: float, phi: float) -> complex:
    """Psi4 at the point of angles (theta, phi) on the sphere |x - centre| = r."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    out = np.empty(2)
    if lib().orc_psi4_point(ctypes.byref(_cp(p)), _ptr(u), _ptr(c), float(r), float(theta), float(phi),
                            _ptr(out)) != 0:
        raise ValueError("stencil leaves the patch")
    return complex(out[0], out[1])


def psi4_modes(p, u: np.ndarray, centre, r: float, ntheta: int = 24, nphi: int = 48, lmax: int = 4):
    """{(l, m): Psi4^lm} for l = 2..lmax on the sphere |x - centre| = r."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    nm = (lmax + 1) ** 2 - 4
    out = np.empty(2 * nm)
    if lib().orc_psi4_modes(ctypes.byref(_cp(p)), _ptr(u), _ptr(c), float(r), int(ntheta), int(nphi), int(lmax),
                            _ptr(out)) != 0:
        raise ValueError("sphere leaves the patch")
    modes = {}
    k = 0
    for l in range(2, lmax + 1):
        for m in range(-l, l + 1):
            modes[(l, m)] = complex(out[2 * k], out[2 * k + 1])
            k += 1
    return modes


def swsh(l: int, m: int, theta: float, phi: float) -> complex:
    out = np.empty(2)
    lib().orc_swsh(int(l), int(m), float(theta), float(phi), _ptr(out))
    return complex(out[0], out[1])


def gauss_legendre(n: int):
    x = np.empty(n)
    w = np.empty(n)
    lib().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def lagrange_weights(nodes: Sequence[int], x: float) -> np.ndarray:
    arr = (ctypes.c_int * len(nodes))(*nodes)
    w = np.empty(len(nodes))
    lib().orc_lagrange_weights(len(nodes), arr, x, _ptr(w))
    return w


def time_weights(nlevels: int, s: float) -> np.ndarray:
    """Weights of the parent time levels (oldest first) at fraction s of the
    parent step measured from the middle level (Sec. 2.2.1: quadratic through
    t-DT, t, t+DT once three levels exist; linear through t, t+DT before)."""
    if nlevels >= 3:
        return lagrange_weights([-1, 0, 1], s)
    return np.concatenate([[0.0], lagrange_weights([0, 1], s)])


# ------------------------------------------------------------------ Berger-Oliger driver

class BOHierarchy:
    """Berger-Oliger subcycling over a static box-in-box hierarchy (Sec. 2.2.1).

    level_step(l): one RK4 step of level l (dt_l = courant * dx_l) with child
    ghosts prolonged (space: 6th-order Lagrange; time: quadratic through the
    parent's three time levels, linear while only two exist) and then exchanged
    between same-level patches at every stage; then two steps of level l+1;
    then, for level l+1: ghosts prolonged at the parent's new time from the
    unrestricted parent, exchange, and restriction of every child onto l.
    Level 0's ghosts follow the Sommerfeld condition and are evolved with the
    stage.  With zsym (equatorial reflection symmetry, Sec. 2.2.2) only z >= 0
    is evolved: the z < 0 ghosts of every patch whose lower face is z = 0 are
    filled by reflection after the other ghost treatments of every stage.
    """

    def __init__(self, hierarchy, states: List[np.ndarray], prm: Params, courant: float = 0.5,
                 bc0: int = BC_SOMMERFELD, previous: Optional[List[np.ndarray]] = None, zsym: bool = False):
        self.h = hierarchy
        self.prm = prm
        self.courant = courant
        self.bc0 = bc0
        self.zsym = zsym
        self.patches = [p for lv in hierarchy.levels for p in lv]
        idx = 0
        self.level_ids = []
        for lv in hierarchy.levels:
            self.level_ids.append(list(range(idx, idx + len(lv))))
            idx += len(lv)
        self.parent = [None] * len(self.patches)
        for l in range(1, len(hierarchy.levels)):
            for pid in self.level_ids[l]:
                self.parent[pid] = self._find_parent(pid, l)
        # time levels per patch: list of arrays, oldest first (at most 3)
        self.tl = [[np.array(s, dtype=np.float64, copy=True)] for s in states]
        if previous is not None:  # states one step dt_l earlier: quadratic interpolation from the start
            for pid, s in enumerate(previous):
                self.tl[pid].insert(0, np.array(s, dtype=np.float64, copy=True))
        self.nsteps = [0] * len(hierarchy.levels)
        self.punct = []                          # puncture positions
        self.follow = [-1] * len(self.patches)   # puncture each patch follows
        self.track_patch = []                    # the patch that tracks each puncture

    def _find_parent(self, pid, l):
        c = self.patches[pid]
        for qid in self.level_ids[l - 1]:
            q = self.patches[qid]
            inside = all(q.origin[d] <= c.origin[d] + 1e-12 and
                         c.origin[d] + c.n[d] * c.dx <= q.origin[d] + q.n[d] * q.dx + 1e-12 for d in range(3))
            if inside:
                return qid
        raise ValueError("patch %d has no parent" % pid)

    def dt(self, l):
        return self.courant * self.h.dx0 / (2 ** l)

    # ---- moving boxes (Sec. 2.2.1) ----

    def track(self, positions, follow):
        """Punctures at `positions`; follow[pid] = the puncture patch pid
        follows (-1: none).  Puncture p is tracked on the finest patch that
        follows it: after every step of that patch, dx/dt = -beta(x) is
        integrated over the step with Heun's method, beta interpolated
        (tricubic) from the step's old and new time levels."""
        self.punct = [np.array(x, dtype=np.float64) for x in positions]
        self.follow = [int(v) for v in follow]
        self.track_patch = []
        for p in range(len(self.punct)):
            best = None
            for pid, q in enumerate(self.follow):
                if q == p and (best is None or self.patches[pid].level > self.patches[best].level):
                    best = pid
            self.track_patch.append(best)

    def _track(self, l):
        for p, pid in enumerate(self.track_patch):
            if pid is None or self.patches[pid].level != l:
                continue
            pa, dt = self.patches[pid], self.dt(l)
            u0, u1 = self.tl[pid][-2], self.tl[pid][-1]
            x = self.punct[p]
            b0 = np.array([interp_point(pa, u0, 19 + d, x) for d in range(3)])
            xs = x - dt * b0
            b1 = np.array([interp_point(pa, u1, 19 + d, xs) for d in range(3)])
            self.punct[p] = x - 0.5 * dt * (b0 + b1)

    def synchronised(self) -> bool:
        return all(self.nsteps[l] == self.nsteps[0] * 2 ** l for l in range(len(self.nsteps)))

    def _children(self, pid):
        return [q for q, par in enumerate(self.parent) if par == pid]

    def _nest_lo(self, c, par, d, off):
        """Smallest offset (parent cells) of child c along d inside par."""
        zlow = self.zsym and d == 2 and touches_equator(c) and touches_equator(par) and off == 0
        return 0 if zlow else 4

    def _active_overlap(self, l) -> bool:
        """Do two patches of level l share active cells?"""
        ids = self.level_ids[l]
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                A, B = self.patches[ids[a]], self.patches[ids[b]]
                off = [int(round((A.origin[d] - B.origin[d]) / A.dx)) for d in range(3)]
                if all(off[d] < B.n[d] and off[d] + A.n[d] > 0 for d in range(3)):
                    return True
        return False

    def _shift_range(self, pid, geoms, kids):
        """Per axis the shifts (parent cells) that keep patch pid nested in
        its parent geoms[parent] and the children `kids` (at their geoms)
        nested in it; under equatorial symmetry no patch moves along z
        (punctures on the equator stay there)."""
        c = geoms[pid]
        par = geoms[self.parent[pid]]
        lo, hi = [], []
        for d in range(3):
            off = int(round((c.origin[d] - par.origin[d]) / par.dx))
            a = self._nest_lo(c, par, d, off) - off
            b = par.n[d] - 4 - c.n[d] // 2 - off
            for kid in kids:
                k = geoms[kid]
                koff = int(round((k.origin[d] - c.origin[d]) / c.dx))
                # the child's offset becomes koff - 2 s
                a = max(a, -((c.n[d] - 4 - k.n[d] // 2 - koff) // 2))
                b = min(b, (koff - self._nest_lo(k, c, d, koff)) // 2)
            if self.zsym and d == 2:
                a = b = 0
            lo.append(a)
            hi.append(b)
        return lo, hi

    def shift_range(self, pid):
        return self._shift_range(pid, self.patches, self._children(pid))

    def _shifted(self, c, shift):
        return dataclasses.replace(c, origin=tuple(c.origin[d] + (2 * int(shift[d])) * c.dx for d in range(3)))

    def _apply_move(self, pid, shift):
        c = self.patches[pid]
        new = self._shifted(c, shift)
        ppid = self.parent[pid]
        skip = self.zsym and touches_equator(c)
        un = move_patch(self.patches[ppid], self.tl[ppid][-1], c, self.tl[pid][-1], new, skip_zlower=skip)
        if skip:
            un = fill_zreflect(new, un)
        self.patches[pid] = new
        for q in self.level_ids[new.level]:
            self.tl[q] = [self.tl[q][-1]]
        self.tl[pid] = [un]
        # where the parent level's patches share active cells, the exchange
        # at the start of each of its steps averages them in its stored time
        # levels, and the older levels the moved patch's ghosts would be
        # interpolated from are no longer those of its last steps: that
        # level's history restarts too
        if self._active_overlap(new.level - 1):
            for q in self.level_ids[new.level - 1]:
                self.tl[q] = [self.tl[q][-1]]

    def move_patch(self, pid, shift):
        """Shift patch pid by shift[d] parent cells (2 shift[d] of its own):
        cells that were active keep their values, the others are prolonged
        from the parent's current time level; the time-level history of the
        patch's level restarts (its older levels no longer cover the patch),
        and so does the parent level's where its patches share active cells.
        The shift must keep the patch and its children nested."""
        if not self.synchronised():
            raise ValueError("levels not synchronised")
        lo, hi = self.shift_range(pid)
        if any(not (lo[d] <= shift[d] <= hi[d]) for d in range(3)):
            raise ValueError("shift breaks the nesting")
        self._apply_move(pid, shift)

    def _targets(self):
        """The position each moving patch follows: its puncture's."""
        return {pid: self.punct[p] for pid, p in enumerate(self.follow) if p >= 0}

    def regrid(self) -> int:
        """Coarse to fine, every patch that follows a puncture moves by
        trunc((x_p - centre) / dx_parent) parent cells per axis (the puncture
        then lies within one parent cell of its centre), clamped so that it
        stays nested in its parent's new position and keeps its children
        that follow no puncture nested.  The whole plan is checked before
        any data moves.  Returns the number of patches moved."""
        if not self.synchronised():
            raise ValueError("levels not synchronised")
        geoms = list(self.patches)
        plan = []
        targets = self._targets()
        for l in range(1, len(self.level_ids)):
            for pid in self.level_ids[l]:
                if pid not in targets:
                    continue
                x = targets[pid]
                c = geoms[pid]
                dxp = 2.0 * c.dx
                s = [int(math.trunc((x[d] - (c.origin[d] + 0.5 * c.n[d] * c.dx)) / dxp)) for d in range(3)]
                fixed_kids = [q for q in self._children(pid) if q not in targets]
                lo, hi = self._shift_range(pid, geoms, fixed_kids)
                if any(lo[d] > hi[d] for d in range(3)):
                    raise ValueError("patch %d cannot stay nested" % pid)
                s = [min(max(s[d], lo[d]), hi[d]) for d in range(3)]
                if any(s):
                    geoms[pid] = self._shifted(c, s)
                    plan.append((pid, s))
        for pid in range(len(geoms)):  # the final configuration nests
            if self.parent[pid] is None:
                continue
            lo, hi = self._shift_range(pid, geoms, self._children(pid))
            if any(not (lo[d] <= 0 <= hi[d]) for d in range(3)):
                raise ValueError("regrid would break the nesting of patch %d" % pid)
        for pid, s in plan:
            self._apply_move(pid, s)
        return len(plan)

    def current(self, pid) -> np.ndarray:
        return self.tl[pid][-1]

    def _fill_child_ghosts(self, pid, u, frac):
        """Prolong parent data at fraction frac of the parent's last step."""
        ppid = self.parent[pid]
        levels = self.tl[ppid]
        # the parent's last step went from levels[-2] to levels[-1]
        w = time_weights(len(levels), frac)
        src = levels[-3:] if len(levels) >= 3 else [levels[-2], levels[-1]]
        ws = w if len(levels) >= 3 else w[1:]
        up = np.zeros_like(src[0])
        for wi, si in zip(ws, src):
            up = up + wi * si
        skip = self.zsym and touches_equator(self.patches[pid])
        return prolong_ghosts(self.patches[ppid], up, self.patches[pid], u, skip_zlower=skip)

    def _reflect(self, ids, arrays):
        if not self.zsym:
            return arrays
        return [fill_zreflect(self.patches[pid], a) if touches_equator(self.patches[pid]) else a
                for pid, a in zip(ids, arrays)]

    def _exchange_level(self, l, arrays):
        ids = self.level_ids[l]
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                exchange(self.patches[ids[a]], arrays[a], self.patches[ids[b]], arrays[b])

    def _rk4_level(self, l, frac0, dfrac):
        """One RK4 step of every patch of level l; frac0/dfrac locate the step
        inside the parent's last step (unused on level 0)."""
        ids = self.level_ids[l]
        dt = self.dt(l)
        un = [self.tl[pid][-1] for pid in ids]
        y = [np.zeros_like(a) for a in un]
        cur = [a.copy() for a in un]
        stage_frac = [0.0, 0.5, 0.5, 1.0]
        evolve_ghosts = (l == 0 and self.bc0 == BC_SOMMERFELD)
        for s in range(1, 5):
            if l == 0 and self.bc0 == BC_PERIODIC:
                cur = [fill_periodic(self.patches[pid], c) for pid, c in zip(ids, cur)]
            if l > 0:
                for a, pid in enumerate(ids):
                    cur[a] = self._fill_child_ghosts(pid, cur[a], frac0 + stage_frac[s - 1] * dfrac)
                if len(ids) > 1:
                    self._exchange_level(l, cur)
            cur = self._reflect(ids, cur)
            if s == 1:  # the stage-1 state, ghosts filled, is the step's u_n
                un = [c.copy() for c in cur]
            out = [np.empty_like(a) for a in un]
            for a, pid in enumerate(ids):
                rk4_stage(self.patches[pid], self.prm, s, dt, evolve_ghosts, cur[a], un[a], y[a], out[a])
            cur = out
        # the new level's z < 0 ghosts mirror its own new values: the
        # children's prolongation reads those parent cells
        cur = self._reflect(ids, cur)
        for a, pid in enumerate(ids):
            if l == 0 and self.bc0 == BC_PERIODIC:
                cur[a] = fill_periodic(self.patches[pid], cur[a])
            self.tl[pid].append(cur[a])
            if len(self.tl[pid]) > 3:
                self.tl[pid].pop(0)
        self._track(l)
        self.nsteps[l] += 1

    def level_step(self, l=0, frac0=0.0, dfrac=1.0):
        self._rk4_level(l, frac0, dfrac)
        if l + 1 < len(self.h.levels):
            self.level_step(l + 1, 0.0, 0.5)
            self.level_step(l + 1, 0.5, 0.5)
            # child ghosts at the parent's new time (from the parent before any
            # restriction), same-level exchange, then restriction of every child
            kids = self.level_ids[l + 1]
            for pid in kids:
                self.tl[pid][-1] = self._fill_child_ghosts(pid, self.tl[pid][-1], 1.0)
            if len(kids) > 1:
                cur = [self.tl[pid][-1] for pid in kids]
                self._exchange_level(l + 1, cur)
            if self.zsym:
                cur = self._reflect(kids, [self.tl[pid][-1] for pid in kids])
                for pid, c in zip(kids, cur):
                    self.tl[pid][-1] = c
            for pid in kids:
                ppid = self.parent[pid]
                self.tl[ppid][-1] = restrict(self.patches[ppid], self.tl[ppid][-1],
                                             self.patches[pid], self.tl[pid][-1])
            if self.zsym:  # the restricted cells next to z = 0 have mirrors among the ghosts
                ids = self.level_ids[l]
                cur = self._reflect(ids, [self.tl[pid][-1] for pid in ids])
                for pid, c in zip(ids, cur):
                    self.tl[pid][-1] = c
