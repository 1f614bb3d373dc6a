"""The C ABI library loads, exports every function include/sacrak.h
declares, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    skbuild.build()
    return sk.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "sacrak.h")).read()
    return sorted(set(re.findall(r"\b(sacrak_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(sk.EXPORTS)


def test_every_declared_symbol_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_arena_bytes_host_side(L):
    import initial_data as idd
    h = idd.binary_7_level()
    def copies(mixed):
        # 6 FP64 state copies per patch (rows padded to a multiple of 8 with at
        # least one spare element), 3 prolongation caches on levels > 0,
        # mixed precision: 5 copies of FP32 hi/lo pairs (= 5 FP64 copies) and
        # 103 FP32 derivative planes over the largest level's 32 x 4 x 1 tiles
        st = sum((6 + (3 if p.level > 0 else 0) + (5 if mixed else 0)) * 25 * 8 *
                 (p.n[0] + 7 + (-(p.n[0] + 7)) % 8) * (p.n[1] + 6) * (p.n[2] + 6) for p in h.patches)
        tiles = max(sum(-(-p.n[0] // 32) * -(-p.n[1] // 4) * p.n[2] for p in lv) for lv in h.levels)
        return st + (103 * 128 * 4 * tiles if mixed else 0)
    n = sk.arena_bytes(len(h.levels), h.patches)
    assert copies(False) <= n < copies(False) + 64 * 2 ** 20
    nm = sk.arena_bytes(len(h.levels), h.patches, sk.Params(precision=1))
    assert copies(True) <= nm < copies(True) + 64 * 2 ** 20
    assert sk.arena_bytes(2, h.patches[:1]) == 0  # level 1 without a patch


def test_invalid_arguments_rejected_before_device_work(L):
    out = ctypes.c_void_p()
    prm = sk.Params().c()
    d = sk._descs([type("P", (), {"level": 0, "n": (8, 8, 8), "origin": (0, 0, 0)})()])
    # null arena
    assert L.sacrak_grid_create(1, 1.0, 1, d, ctypes.byref(prm), None, None, 0, ctypes.byref(out)) == sk.EINVAL
    # bad dx0
    assert L.sacrak_grid_create(1, -1.0, 1, d, ctypes.byref(prm), None, ctypes.c_void_p(256), 1 << 30,
                                ctypes.byref(out)) == sk.EINVAL
    # null grid handles
    assert L.sacrak_rk4_step(None, 0, 0.1) == sk.EINVAL
    assert L.sacrak_level_step(None, 0) == sk.EINVAL
    assert L.sacrak_grid_destroy(None) == sk.EINVAL
    assert L.sacrak_last_error(None) == b"null grid"


def test_diagnostics_and_moving_boxes_reject_before_device_work(L):
    """The newer entry points validate their handles and arguments on the
    host: null grids, null arrays and impossible parameters return
    SACRAK_EINVAL without touching a device."""
    d = ctypes.c_double
    c3 = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    out = (ctypes.c_double * 160)()
    assert L.sacrak_adm_integrals(None, 0, c3, d(1.0), 8, 16, out) == sk.EINVAL
    assert L.sacrak_psi4_modes(None, 0, c3, d(1.0), 8, 16, 2, out) == sk.EINVAL
    assert L.sacrak_track_punctures(None, 0, None, None) == sk.EINVAL
    assert L.sacrak_get_punctures(None, out) == sk.EINVAL
    assert L.sacrak_move_patch(None, 0, (ctypes.c_int * 3)(1, 0, 0)) == sk.EINVAL
    assert L.sacrak_regrid(None, ctypes.byref(ctypes.c_int())) == sk.EINVAL
    assert L.sacrak_patch_origin(None, 0, c3) == sk.EINVAL
    assert L.sacrak_density_maximum(None, 0, out) == sk.EINVAL
    assert L.sacrak_track_stars(None, 0, None) == sk.EINVAL
    # waveform post-processing: null arrays, n < 1, l < 2, r0 = m0 / 2
    # (D0 / (2 m0) = 1), non-positive spacing or cut
    p = ctypes.c_void_p(256)
    assert L.sacrak_nakano(None, p, 8, 2, d(100.0), d(1.0), p, p, None) == sk.EINVAL
    assert L.sacrak_nakano(p, p, 0, 2, d(100.0), d(1.0), p, p, None) == sk.EINVAL
    assert L.sacrak_nakano(p, p, 8, 1, d(100.0), d(1.0), p, p, None) == sk.EINVAL
    assert L.sacrak_nakano(p, p, 8, 2, d(1.0), d(2.0), p, p, None) == sk.EINVAL
    assert L.sacrak_ffi_strain(None, 8, d(0.1), d(0.5), p, p, ctypes.c_size_t(1 << 20), None) == sk.EINVAL
    assert L.sacrak_ffi_strain(p, 8, d(0.0), d(0.5), p, p, ctypes.c_size_t(1 << 20), None) == sk.EINVAL
    assert L.sacrak_ffi_strain(p, 8, d(0.1), d(-1.0), p, p, ctypes.c_size_t(1 << 20), None) == sk.EINVAL
    assert L.sacrak_ffi_work_bytes(0) == 0


def test_missing_library_fails_loudly(monkeypatch):
    """Without libsacrak.so the binding raises: there is no fallback path."""
    monkeypatch.setattr(sk, "_lib", None)
    monkeypatch.setattr(sk, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libsacrak.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sk.lib()


def test_arena_bytes_with_a_fluid(L):
    """A fluid adds 107 arrays of the patch layout (conserved variables in the
    six state slots, primitives with the Lorentz factor, face fluxes, Z4c
    matter terms, the cached prolongations of the parent's three time levels
    and the two sets of RK4-weighted face fluxes for the reflux); it needs
    FP64 and no overlapping patches on a level."""
    import initial_data as idd
    p = idd.centred_patch(24, 0.5)
    n0 = sk.arena_bytes(1, [p], sk.Params())
    n1 = sk.arena_bytes(1, [p], sk.Params(matter=1))
    fs = (p.n[0] + 7 + (-(p.n[0] + 7)) % 8) * (p.n[1] + 6) * (p.n[2] + 6)
    assert 107 * 8 * fs <= n1 - n0 < 107 * 8 * fs + 512
    assert sk.arena_bytes(1, [p], sk.Params(matter=1, precision=1)) == 0
    h = idd.binary_7_level()
    assert sk.arena_bytes(len(h.levels), h.patches, sk.Params(matter=1)) > 0
