"""Waveform post-processing on the GPU (Sec. 2.3): Nakano extrapolation and
fixed frequency integration against the oracle (1e-12 of the largest value:
the scan and the FFT sum in other orders), on ragged lengths (not multiples
of the 1024-thread scan, fewer samples than threads, a non-power-of-two FFT
length), on non-uniform sample times, and the oracle-pinned closed forms;
argument errors."""
import ctypes
import math

import numpy as np
import pytest

from oracle import waveform

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

skbuild.build()


def _series(n, seed=2, uniform=True):
    rng = np.random.default_rng(seed)
    t = np.linspace(10.0, 410.0, n) if uniform else np.sort(rng.uniform(10.0, 410.0, n))
    ph = 0.05 * t + 2e-4 * t * t
    psi = (1e-3 + 1e-5 * t) * np.exp(-1j * ph) + 1e-6 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    return t, psi


@pytest.mark.parametrize("n,uniform,l", [(10007, True, 2), (5, True, 3), (1, True, 2), (4096, False, 4)])
def test_nakano_parity(n, uniform, l):
    t, psi = _series(n, uniform=uniform)
    tg, og = sk.nakano_extrapolate(t, psi, l, 120.0, 2.8)
    to, oo = waveform.nakano_extrapolate(t, psi, l, 120.0, 2.8)
    assert np.abs(tg - to).max() <= 1e-12 * np.abs(to).max()
    assert np.abs(og - oo).max() <= 1e-12 * np.abs(oo).max()


def test_nakano_closed_form_integral():
    A, w, l, r0, m0 = 0.3 + 0.1j, 0.7, 3, 100.0, 2.7
    t = np.linspace(5.0, 65.0, 4000)
    psi = A * np.exp(-1j * w * t)
    _, out = sk.nakano_extrapolate(t, psi, l, r0, m0)
    d0 = 102.718225
    integ = A * (np.exp(-1j * w * t) - np.exp(-1j * w * t[0])) / (-1j * w)
    assert np.abs(out - (1.0 - 5.4 / d0) * (d0 * psi - 5.0 * integ)).max() < 1e-4


@pytest.mark.parametrize("n", [4096, 3001])
def test_ffi_parity(n):
    t, psi = _series(n)
    dt = t[1] - t[0]
    hg = sk.ffi_strain(psi, dt, 0.01)
    ho = waveform.ffi_strain(psi, dt, 0.01)
    assert np.abs(hg - ho).max() <= 1e-12 * np.abs(ho).max()


def test_ffi_closed_form():
    n, dt = 4096, 0.05
    T = n * dt
    t = np.arange(n) * dt
    w1 = 2 * math.pi * 40 / T
    wl = 2 * math.pi * 3 / T
    h = 0.2 * np.exp(-1j * w1 * t)
    low = 0.1 * np.exp(-1j * wl * t)
    psi = w1 ** 2 * h + wl ** 2 * low
    out = sk.ffi_strain(psi, dt, 10 / T)
    assert np.abs(out - (h + low * (wl * T / (2 * math.pi * 10)) ** 2)).max() < 1e-12


def test_errors():
    L = sk.lib()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = torch.zeros(16, dtype=torch.float64, device="cuda")
    o = torch.zeros(16, dtype=torch.float64, device="cuda")
    v = lambda x: ctypes.c_void_p(x.data_ptr())
    d = ctypes.c_double
    assert L.sacrak_nakano(v(t), v(p), 8, 1, d(100.0), d(2.0), v(t), v(o), None) == 1  # l < 2
    assert L.sacrak_nakano(v(t), v(p), 8, 2, d(1.0), d(2.0), v(t), v(o), None) == 1   # D0 / 2 m0 = 1
    assert L.sacrak_nakano(v(t), v(p), 0, 2, d(100.0), d(2.0), v(t), v(o), None) == 1
    wb = L.sacrak_ffi_work_bytes(8)
    assert wb > 0
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    assert L.sacrak_ffi_strain(v(p), 8, d(0.1), d(0.0), v(o), v(work), ctypes.c_size_t(wb), None) == 1
    if wb > 1:
        assert L.sacrak_ffi_strain(v(p), 8, d(0.1), d(0.5), v(o), v(work), ctypes.c_size_t(wb - 1), None) == 1
    assert L.sacrak_ffi_strain(v(p), 8, d(0.1), d(0.5), v(o), v(work), ctypes.c_size_t(wb), None) == 0
