"""Python binding of libsacrak (the C ABI in include/sacrak.h).

Argument marshalling only: every step of the Z4c hot path runs in the CUDA
kernels of libsacrak.so.  PyTorch provides the device arena and the stream.
There is no CPU fallback: importing works without a GPU, but creating a grid
needs the built library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsacrak.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE = range(7)
_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENONFINITE", "ETIMEOUT", "ESTATE"]
NF = 25
GHOST = 3

# functions the header declares (checked by the ABI test)
EXPORTS = [
    "sacrak_arena_bytes", "sacrak_grid_create", "sacrak_grid_destroy", "sacrak_set_initial_data",
    "sacrak_upload_fields", "sacrak_download_fields", "sacrak_rhs", "sacrak_rk4_step",
    "sacrak_level_step", "sacrak_constraints", "sacrak_pi_symmetry", "sacrak_level_time",
    "sacrak_last_error", "sacrak_profile_enable", "sacrak_profile_read", "sacrak_constraints_noalloc",
    "sacrak_set_stage_kernel", "sacrak_get_stage_kernel", "sacrak_autotune", "sacrak_adm_integrals",
    "sacrak_track_punctures", "sacrak_get_punctures", "sacrak_move_patch", "sacrak_regrid",
    "sacrak_patch_origin", "sacrak_psi4_modes", "sacrak_nakano", "sacrak_ffi_work_bytes", "sacrak_ffi_strain",
    "sacrak_set_wait_limit", "sacrak_set_eos", "sacrak_set_atmosphere", "sacrak_upload_matter",
    "sacrak_download_matter", "sacrak_matter_rhs", "sacrak_set_overlap", "sacrak_set_riemann",
    "sacrak_density_maximum", "sacrak_track_stars",
]

# stage kernels (sacrak_set_stage_kernel): 0 direct, 1..4 TMA-staged tiles,
# 5..6 L1 path with packed pair arithmetic (without / with prefetching),
# 7 split into a derivative and an algebra launch, 8 as 6 with 4 CTAs per SM,
# 9 as 6 prefetching the star rows only, 10 only the z-arm rows, 11 only the
# RK update's streaming reads, 12 as 10 with the x-neighbour inner differences
# of the mixed derivatives exchanged by warp shuffles, 13 as 12 with 4 CTAs per SM,
# 14 as 10 with 4 CTAs per SM, 15 two x-adjacent points per thread with 128-bit
# loads of the hi/lo pairs, 16 as 15 prefetching the next field's z-arm rows,
# 17 as 16 with 3 CTAs per SM (more of the SM's memory left to L1), 18 as 10
# with a persistent grid (resident CTAs walk the level's tiles)
STAGE_KERNELS = {0: "direct", 1: "tma 32x4x1", 2: "tma 32x2x2", 3: "tma 32x4x2", 4: "tma 32x8x1",
                 5: "l1 pairs", 6: "l1 pairs + prefetch", 7: "split deriv + algebra",
                 8: "l1 pairs + prefetch, 4/SM", 9: "l1 pairs + star prefetch",
                 10: "l1 pairs + z-arm prefetch", 11: "l1 pairs + epilogue prefetch",
                 12: "l1 pairs + z-arm prefetch + x shuffles", 13: "l1 pairs + z-arm prefetch + x shuffles, 4/SM",
                 14: "l1 pairs + z-arm prefetch, 4/SM", 15: "two points/thread, 128-bit loads",
                 16: "two points/thread, 128-bit loads + z-arm prefetch",
                 17: "two points/thread, 128-bit loads + z-arm prefetch, 3/SM",
                 18: "l1 pairs + z-arm prefetch, persistent",
                 19: "l1 pairs + z-arm prefetch, compile-time pitches",
                 20: "l1 pairs + z-arm prefetch, compile-time pitches, 4/SM (default)"}


class SacrakError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class sacrak_params(ctypes.Structure):
    _fields_ = [("kappa1", ctypes.c_double), ("kappa2", ctypes.c_double), ("eta", ctypes.c_double),
                ("sigma_ko", ctypes.c_double), ("courant", ctypes.c_double), ("w_floor", ctypes.c_double),
                ("lapse", ctypes.c_int), ("shift", ctypes.c_int), ("bc", ctypes.c_int),
                ("precision", ctypes.c_int), ("lapse_uses_khat", ctypes.c_int), ("zsym", ctypes.c_int),
                ("matter", ctypes.c_int)]


class sacrak_patch_desc(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("n", ctypes.c_int * 3), ("origin", ctypes.c_double * 3)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libsacrak.so (build it first with paper_2607_08743_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsacrak.so is not built (%s); run paper_2607_08743_gb300.build.build()"
                                   % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            vp, dp = ctypes.c_void_p, P(ctypes.c_double)
            L.sacrak_arena_bytes.restype = ctypes.c_size_t
            L.sacrak_arena_bytes.argtypes = [ctypes.c_int, ctypes.c_int, P(sacrak_patch_desc), P(sacrak_params)]
            L.sacrak_grid_create.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             P(sacrak_patch_desc), P(sacrak_params), vp, vp,
                                             ctypes.c_size_t, P(vp)]
            L.sacrak_grid_destroy.argtypes = [vp]
            L.sacrak_set_initial_data.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                  ctypes.c_int]
            L.sacrak_upload_fields.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_download_fields.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_rhs.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_rk4_step.argtypes = [vp, ctypes.c_int, ctypes.c_double]
            L.sacrak_level_step.argtypes = [vp, ctypes.c_int]
            L.sacrak_constraints.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp]
            L.sacrak_pi_symmetry.argtypes = [vp, ctypes.c_int, dp]
            L.sacrak_level_time.argtypes = [vp, ctypes.c_int, dp]
            L.sacrak_profile_enable.argtypes = [vp, ctypes.c_int]
            L.sacrak_profile_read.argtypes = [vp, dp, P(ctypes.c_longlong), P(ctypes.c_longlong)]
            L.sacrak_constraints_noalloc.argtypes = [vp, P(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                                     vp, dp]
            L.sacrak_set_stage_kernel.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.sacrak_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
            L.sacrak_set_overlap.argtypes = [vp, ctypes.c_int]
            L.sacrak_set_riemann.argtypes = [vp, ctypes.c_int]
            L.sacrak_set_eos.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_double]
            L.sacrak_set_atmosphere.argtypes = [vp, ctypes.c_double, ctypes.c_double]
            L.sacrak_upload_matter.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_download_matter.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_matter_rhs.argtypes = [vp, ctypes.c_int, vp]
            L.sacrak_density_maximum.argtypes = [vp, ctypes.c_int, dp]
            L.sacrak_track_stars.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
            L.sacrak_get_stage_kernel.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
            L.sacrak_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
            L.sacrak_last_error.argtypes = [vp]
            L.sacrak_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("sacrak_arena_bytes", "sacrak_last_error", "sacrak_ffi_work_bytes"):
                    getattr(L, name).restype = ctypes.c_int
            L.sacrak_ffi_work_bytes.argtypes = [ctypes.c_int]
            L.sacrak_ffi_work_bytes.restype = ctypes.c_size_t
            _lib = L
    return _lib


@dataclasses.dataclass
class Params:
    """sacrak_params; defaults are the paper's (Sec. 2.2, Sec. 3)."""
    kappa1: float = 0.005
    kappa2: float = 0.0
    eta: float = 0.36
    sigma_ko: float = 0.5
    courant: float = 0.5
    w_floor: float = 1e-10
    lapse: int = 0
    shift: int = 0
    bc: int = 0            # 0 Sommerfeld, 1 periodic, 2 frozen
    precision: int = 0     # 0 FP64, 1 mixed
    lapse_uses_khat: int = 0
    zsym: int = 0          # 1: equatorial reflection symmetry, only z >= 0 evolved
    matter: int = 0        # 1: a perfect fluid evolved with the spacetime (FP64)

    def c(self) -> sacrak_params:
        return sacrak_params(self.kappa1, self.kappa2, self.eta, self.sigma_ko, self.courant, self.w_floor,
                             self.lapse, self.shift, self.bc, self.precision, self.lapse_uses_khat,
                             self.zsym, self.matter)


def _descs(patches) -> ctypes.Array:
    arr = (sacrak_patch_desc * len(patches))()
    for i, p in enumerate(patches):
        arr[i].level = int(getattr(p, "level", 0))
        for d in range(3):
            arr[i].n[d] = int(p.n[d])
            arr[i].origin[d] = float(p.origin[d])
    return arr


def arena_bytes(nlevels: int, patches, params: Optional["Params"] = None) -> int:
    d = _descs(patches)
    prm = params.c() if params is not None else None
    return int(lib().sacrak_arena_bytes(nlevels, len(patches), d, ctypes.byref(prm) if prm else None))


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise SacrakError(EINVAL, "expected a C-contiguous float64 array")
        return a.ctypes.data
    import torch
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise SacrakError(EINVAL, "expected a contiguous float64 tensor")
    return a.data_ptr()


def nakano_extrapolate(t, psi, l: int, r0: float, m0: float, stream=None):
    """(t_ret, D0 Psi4^{l,m,inf}) of one mode's time series (Sec. 2.3), on
    the GPU (numpy in, numpy out)."""
    import torch
    tt = torch.as_tensor(np.ascontiguousarray(t, dtype=np.float64), device="cuda")
    pc = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
    pp = torch.as_tensor(pc.view(np.float64).copy(), device="cuda")
    tr = torch.empty_like(tt)
    out = torch.empty_like(pp)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().sacrak_nakano(ctypes.c_void_p(tt.data_ptr()), ctypes.c_void_p(pp.data_ptr()), len(tt), int(l),
                             ctypes.c_double(r0), ctypes.c_double(m0), ctypes.c_void_p(tr.data_ptr()),
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise SacrakError(st, "sacrak_nakano failed")
    s.synchronize()
    return tr.cpu().numpy(), out.cpu().numpy().view(np.complex128)


def ffi_strain(psi, dt: float, f_cut: float, stream=None):
    """Strain h = h_+ - i h_x of a uniformly sampled Psi4 mode by fixed
    frequency integration (Sec. 2.3), on the GPU."""
    import torch
    pc = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
    pp = torch.as_tensor(pc.view(np.float64).copy(), device="cuda")
    h = torch.empty_like(pp)
    n = len(pc)
    wb = lib().sacrak_ffi_work_bytes(n)
    if wb == 0:
        raise SacrakError(3, "cuFFT not available")
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().sacrak_ffi_strain(ctypes.c_void_p(pp.data_ptr()), n, ctypes.c_double(dt), ctypes.c_double(f_cut),
                                 ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                 ctypes.c_size_t(wb), ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise SacrakError(st, "sacrak_ffi_strain failed")
    return h.cpu().numpy().view(np.complex128)


def constraints_noalloc(dev_u, n, dx: float, w_excise: float = 0.0, stream=None) -> np.ndarray:
    """Constraint norms of one patch array held in caller-owned device memory
    (a CUDA tensor in the unpadded patch-array layout), without a grid and
    without any device allocation (sacrak_constraints_noalloc)."""
    import torch
    nn = [int(v) for v in n]
    if len(nn) != 3:
        raise SacrakError(EINVAL, "n must hold 3 sizes")
    if not isinstance(dev_u, torch.Tensor) or not dev_u.is_cuda:
        raise SacrakError(EINVAL, "dev_u must be a CUDA tensor")
    if dev_u.dtype != torch.float64 or not dev_u.is_contiguous():
        raise SacrakError(EINVAL, "dev_u must be a contiguous float64 tensor")
    if dev_u.device.index != torch.cuda.current_device():
        raise SacrakError(EINVAL, "dev_u is not on the current CUDA device")
    need = NF * (nn[0] + 6) * (nn[1] + 6) * (nn[2] + 6)
    if min(nn) < 1 or dev_u.numel() < need:
        raise SacrakError(EINVAL, "dev_u holds %d values, the patch array needs %d" % (dev_u.numel(), need))
    out = np.empty(4)
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = lib().sacrak_constraints_noalloc(ctypes.c_void_p(dev_u.data_ptr()), (ctypes.c_int * 3)(*nn), dx,
                                          w_excise, sp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise SacrakError(st, "sacrak_constraints_noalloc failed")
    return out


class Grid:
    """A static box-in-box hierarchy on one GPU.  `patches` are objects with
    .level, .n (3 ints) and .origin (3 floats); level l has spacing dx0/2^l."""

    def __init__(self, nlevels: int, dx0: float, patches: Sequence, params: Params = Params(),
                 stream=None, device=None):
        import torch
        self._torch = torch
        L = lib()
        self.nlevels = nlevels
        self.dx0 = dx0
        self.patches = list(patches)
        self.params = params
        d = _descs(self.patches)
        prm0 = params.c()
        nbytes = L.sacrak_arena_bytes(nlevels, len(self.patches), d, ctypes.byref(prm0))
        if nbytes == 0:
            raise SacrakError(EINVAL, "invalid patch description")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            self.arena = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            h = ctypes.c_void_p()
            prm = params.c()
            st = L.sacrak_grid_create(nlevels, dx0, len(self.patches), d, ctypes.byref(prm),
                                      ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.c_void_p(self.arena.data_ptr()), nbytes, ctypes.byref(h))
        if st != OK:
            raise SacrakError(st, "sacrak_grid_create failed")
        self._h = h
        self.arena_bytes = nbytes

    # ------------------------------------------------------------------ helpers
    def _check(self, st: int, what: str):
        if st != OK:
            msg = lib().sacrak_last_error(self._h).decode()
            raise SacrakError(st, "%s: %s" % (what, msg))

    def shape(self, patch: int):
        p = self.patches[patch]
        return (NF, p.n[2] + 2 * GHOST, p.n[1] + 2 * GHOST, p.n[0] + 2 * GHOST)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sacrak_grid_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ ABI
    def set_initial_data(self, kind: int = 0, masses=(), positions=(), gw_amp: float = 0.0,
                         gw_len: float = 1.0, noise_amp: float = 0.0, seed: int = 0,
                         symmetrise_pi: bool = False):
        m = np.ascontiguousarray(masses, dtype=np.float64)
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.float64).reshape(-1))
        dp = ctypes.POINTER(ctypes.c_double)
        st = lib().sacrak_set_initial_data(self._h, kind, len(m), m.ctypes.data_as(dp) if len(m) else None,
                                           pos.ctypes.data_as(dp) if len(pos) else None, gw_amp, gw_len,
                                           noise_amp, seed, int(symmetrise_pi))
        self._check(st, "set_initial_data")

    def upload_fields(self, patch: int, data):
        if isinstance(data, np.ndarray):
            data = np.ascontiguousarray(data, dtype=np.float64)
            assert data.shape == self.shape(patch)
        self._check(lib().sacrak_upload_fields(self._h, patch, ctypes.c_void_p(_ptr(data))), "upload_fields")

    def download_fields(self, patch: int, out=None):
        if out is None:
            out = np.empty(self.shape(patch))
        self._check(lib().sacrak_download_fields(self._h, patch, ctypes.c_void_p(_ptr(out))), "download_fields")
        return out

    def rhs(self, patch: int, out=None):
        if out is None:
            out = np.empty(self.shape(patch))
        self._check(lib().sacrak_rhs(self._h, patch, ctypes.c_void_p(_ptr(out))), "rhs")
        return out

    # ---- matter (Sec. 2.1.2, 2.2) ----

    def matter_shape(self, patch: int):
        sh = self.shape(patch)
        return (5,) + tuple(sh[1:])

    def set_eos(self, K0: float, gammas, rho_bounds=(), gamma_th: float = 1.8):
        """Hybrid EOS: piecewise polytrope (K0, gammas, rho_bounds) + thermal part."""
        g = (ctypes.c_double * len(gammas))(*[float(v) for v in gammas])
        b = (ctypes.c_double * max(1, len(rho_bounds)))(*[float(v) for v in rho_bounds])
        self._check(lib().sacrak_set_eos(self._h, len(gammas), float(K0), g, b, float(gamma_th)), "set_eos")

    def set_riemann(self, solver: str = "hllc"):
        """Face flux of the fluid: "hllc" (HLLC in the face tetrad, HLLE
        where its intermediate state is unphysical; the default) or "hlle"
        (HLLE in the coordinate frame)."""
        code = {"hllc": 0, "hlle": 1}.get(solver)
        if code is None:
            raise SacrakError(EINVAL, "solver must be 'hllc' or 'hlle'")
        self._check(lib().sacrak_set_riemann(self._h, code), "set_riemann")

    def set_atmosphere(self, rho_atm: float, r_atm: float):
        self._check(lib().sacrak_set_atmosphere(self._h, float(rho_atm), float(r_atm)), "set_atmosphere")

    def upload_matter(self, patch: int, prim):
        if isinstance(prim, np.ndarray):
            prim = np.ascontiguousarray(prim, dtype=np.float64)
            if prim.shape != self.matter_shape(patch):
                raise SacrakError(EINVAL, "matter array of shape %s, expected %s" % (prim.shape, self.matter_shape(patch)))
        self._check(lib().sacrak_upload_matter(self._h, patch, ctypes.c_void_p(_ptr(prim))), "upload_matter")

    def download_matter(self, patch: int, out=None):
        if out is None:
            out = np.empty(self.matter_shape(patch))
        self._check(lib().sacrak_download_matter(self._h, patch, ctypes.c_void_p(_ptr(out))), "download_matter")
        return out

    def matter_rhs(self, patch: int, out=None):
        if out is None:
            out = np.empty(self.matter_shape(patch))
        self._check(lib().sacrak_matter_rhs(self._h, patch, ctypes.c_void_p(_ptr(out))), "matter_rhs")
        return out

    def rk4_step(self, level: int = 0, dt: float = 0.0):
        self._check(lib().sacrak_rk4_step(self._h, level, dt), "rk4_step")

    def level_step(self, level: int = 0):
        self._check(lib().sacrak_level_step(self._h, level), "level_step")

    def constraints(self, level: int = 0, w_excise: float = 0.0) -> np.ndarray:
        out = np.empty(4)
        self._check(lib().sacrak_constraints(self._h, level, w_excise,
                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "constraints")
        return out

    def track_punctures(self, positions, follow):
        """Track punctures at `positions` (N x 3); follow[patch] = puncture
        the patch follows (-1: none)."""
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.float64).reshape(-1))
        n = pos.size // 3
        fl = (ctypes.c_int * max(1, len(follow)))(*[int(v) for v in follow])
        pp = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(lib().sacrak_track_punctures(self._h, n, pp, fl), "track_punctures")
        self._npunct = n

    def punctures(self) -> np.ndarray:
        n = getattr(self, "_npunct", 0)
        out = np.zeros(3 * max(1, n))
        self._check(lib().sacrak_get_punctures(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "get_punctures")
        return out[:3 * n].reshape(n, 3)

    def move_patch(self, patch: int, shift):
        sh = (ctypes.c_int * 3)(*[int(v) for v in shift])
        self._check(lib().sacrak_move_patch(self._h, patch, sh), "move_patch")

    def patch_origin(self, patch: int):
        o = (ctypes.c_double * 3)()
        self._check(lib().sacrak_patch_origin(self._h, patch, o), "patch_origin")
        return tuple(o)

    def density_maximum(self, patch: int):
        """(rho_max, x, y, z) over the patch's active cells (fluid grids)."""
        out = (ctypes.c_double * 4)()
        self._check(lib().sacrak_density_maximum(self._h, patch, out), "density_maximum")
        return tuple(out)

    def track_stars(self, follow):
        """follow[patch] = the star the patch follows (-1: none); regrid()
        moves the followers toward each star's density maximum."""
        n = max([int(v) for v in follow] + [-1]) + 1
        fl = (ctypes.c_int * max(1, len(follow)))(*[int(v) for v in follow])
        self._check(lib().sacrak_track_stars(self._h, n, fl), "track_stars")

    def regrid(self) -> int:
        m = ctypes.c_int()
        self._check(lib().sacrak_regrid(self._h, ctypes.byref(m)), "regrid")
        return m.value

    def adm_integrals(self, patch: int, centre=(0.0, 0.0, 0.0), radius: float = 1.0, ntheta: int = 24,
                      nphi: int = 48):
        """(M_ADM, J_z, P_x, P_y, P_z) on the sphere |x - centre| = radius of
        the patch."""
        c = (ctypes.c_double * 3)(*[float(v) for v in centre])
        out = (ctypes.c_double * 5)()
        self._check(lib().sacrak_adm_integrals(self._h, patch, c, ctypes.c_double(radius), ntheta, nphi, out),
                    "adm_integrals")
        return tuple(float(v) for v in out)

    def psi4_modes(self, patch: int, centre=(0.0, 0.0, 0.0), radius: float = 1.0, ntheta: int = 24,
                   nphi: int = 48, lmax: int = 4):
        """{(l, m): Psi4^lm} on the sphere |x - centre| = radius of the patch."""
        c = (ctypes.c_double * 3)(*[float(v) for v in centre])
        nm = (lmax + 1) ** 2 - 4
        out = (ctypes.c_double * (2 * max(nm, 1)))()
        self._check(lib().sacrak_psi4_modes(self._h, patch, c, ctypes.c_double(radius), ntheta, nphi, lmax, out),
                    "psi4_modes")
        modes, k = {}, 0
        for l in range(2, lmax + 1):
            for m in range(-l, l + 1):
                modes[(l, m)] = complex(out[2 * k], out[2 * k + 1])
                k += 1
        return modes

    def pi_symmetry(self, patch: int = 0) -> float:
        v = ctypes.c_double()
        self._check(lib().sacrak_pi_symmetry(self._h, patch, ctypes.byref(v)), "pi_symmetry")
        return v.value

    def level_time(self, level: int = 0) -> float:
        v = ctypes.c_double()
        self._check(lib().sacrak_level_time(self._h, level, ctypes.byref(v)), "level_time")
        return v.value

    def profile_enable(self, enable: bool = True):
        self._check(lib().sacrak_profile_enable(self._h, int(enable)), "profile_enable")

    def profile_read(self):
        """(summed stage-kernel ms, launches, zones updated) since enabling."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        z = ctypes.c_longlong()
        self._check(lib().sacrak_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(z)),
                    "profile_read")
        return ms.value, n.value, z.value

    def set_stage_kernel(self, level: int, kernel: int):
        """Stage kernel of a level (see STAGE_KERNELS)."""
        self._check(lib().sacrak_set_stage_kernel(self._h, level, kernel), "set_stage_kernel")

    def set_wait_limit(self, cycles: int):
        """Bound (SM cycles) of the TMA stage kernels' copy waits; 0 = default,
        < 0 = run out at once (tests of the time-out path)."""
        self._check(lib().sacrak_set_wait_limit(self._h, int(cycles)), "set_wait_limit")

    def set_overlap(self, on: bool):
        """Refined levels' ghost fills and prolongation beside the stage
        kernels on a second stream (default) or all on the grid's stream."""
        self._check(lib().sacrak_set_overlap(self._h, 1 if on else 0), "set_overlap")

    def stage_kernel(self, level: int) -> int:
        v = ctypes.c_int()
        self._check(lib().sacrak_get_stage_kernel(self._h, level, ctypes.byref(v)), "get_stage_kernel")
        return v.value

    def autotune(self, reps: int = 3, use_cache: bool = True) -> np.ndarray:
        """Time every usable stage kernel on every level and keep the fastest;
        returns the timings (nlevels x len(STAGE_KERNELS), microseconds per launch, -1 = not
        timed) and leaves the choice in place."""
        out = np.full((self.nlevels, len(STAGE_KERNELS)), -1.0)
        self._check(lib().sacrak_autotune(self._h, reps, int(use_cache),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "autotune")
        return out

    def last_error(self) -> str:
        return lib().sacrak_last_error(self._h).decode()
