"""Waveform post-processing of the Psi4 modes (Sec. 2.3) -- oracle, test
infrastructure only (plain numpy, FP64).

* nakano_extrapolate: the retarded time t_ret = t - [D0 + 2 m0 ln(D0 / (2 m0)
  - 1)] and D0 Psi4^{lm,inf} = C(r0) [D0 Psi4^lm(t, r0) - (l-1)(l+2)/2
  int_{t_0}^t Psi4^lm dt'] with D0 = r0 (1 + m0 / (2 r0))^2, C = 1 - 2 m0 / D0;
  the time integral by the trapezoid rule from the first sample.
* ffi_strain: h = IFFT[ FFT(Psi4) / (2 pi max(|f|, f_cut))^2 ] over the DFT
  frequencies of the uniformly sampled series (fixed frequency integration;
  h = h_+ - i h_x = -int int Psi4 for frequencies above f_cut).
"""
from __future__ import annotations

import math

import numpy as np


def nakano_extrapolate(t: np.ndarray, psi: np.ndarray, l: int, r0: float, m0: float):
    """Returns (t_ret, D0 Psi4^{l,m,inf}) for one mode's time series."""
    t = np.asarray(t, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.complex128)
    d0 = r0 * (1.0 + m0 / (2.0 * r0)) ** 2
    c = 1.0 - 2.0 * m0 / d0
    t_ret = t - (d0 + 2.0 * m0 * math.log(d0 / (2.0 * m0) - 1.0))
    integral = np.zeros_like(psi)
    for n in range(1, len(t)):  # trapezoid rule, sample by sample
        integral[n] = integral[n - 1] + 0.5 * (t[n] - t[n - 1]) * (psi[n] + psi[n - 1])
    return t_ret, c * (d0 * psi - 0.5 * (l - 1) * (l + 2) * integral)


def ffi_strain(psi: np.ndarray, dt: float, f_cut: float) -> np.ndarray:
    psi = np.asarray(psi, dtype=np.complex128)
    f = np.fft.fftfreq(len(psi), dt)
    return np.fft.ifft(np.fft.fft(psi) / (2.0 * math.pi * np.maximum(np.abs(f), f_cut)) ** 2)
