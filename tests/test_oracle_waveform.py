"""Pins of the waveform post-processing oracle (Sec. 2.3).

* Nakano extrapolation on Psi4 = A exp(-i w t): the time integral has the
  closed form A (exp(-i w t) - exp(-i w t0)) / (-i w); the result must equal
  C [D0 Psi4 - (l-1)(l+2)/2 int] with that integral to the trapezoid error
  (second order in dt); D0 = r0 (1 + m0/2r0)^2 and t_ret are checked for
  r0 = 100, m0 = 2.7 against their values written out by hand.
* FFI: for h = A exp(-i w t) + B exp(-i 2 w t) with whole periods in the
  window, Psi4 = -d_t^2 h, frequencies above f_cut come back exactly
  (spectral); a component below f_cut comes back scaled by (f / f_cut)^2.
"""
import math

import numpy as np

from oracle import waveform


def test_nakano_against_closed_form_integral():
    A, w, l, r0, m0 = 0.3 + 0.1j, 0.7, 3, 100.0, 2.7
    errs = []
    for n in (2000, 4000):
        t = np.linspace(5.0, 65.0, n)
        psi = A * np.exp(-1j * w * t)
        t_ret, out = waveform.nakano_extrapolate(t, psi, l, r0, m0)
        integ = A * (np.exp(-1j * w * t) - np.exp(-1j * w * t[0])) / (-1j * w)
        d0 = 100.0 * (1.0 + 2.7 / 200.0) ** 2  # 102.718225
        assert abs(d0 - 102.718225) < 1e-9
        c = 1.0 - 5.4 / d0
        exp = c * (d0 * psi - 5.0 * integ)  # (l-1)(l+2)/2 = 5 for l = 3
        errs.append(np.abs(out - exp).max())
        assert abs(t_ret[0] - (5.0 - (d0 + 5.4 * math.log(d0 / 5.4 - 1.0)))) < 1e-12
    assert errs[1] < 1e-4 and 3.5 < errs[0] / errs[1] < 4.5, errs


def test_ffi_exact_above_cut_and_scaled_below():
    n, dt = 4096, 0.05
    T = n * dt
    t = np.arange(n) * dt
    w1 = 2 * math.pi * 40 / T  # whole periods in the window
    w2 = 2 * w1
    wl = 2 * math.pi * 3 / T   # below the cut
    h = 0.2 * np.exp(-1j * w1 * t) + 0.05j * np.exp(-1j * w2 * t)
    low = 0.1 * np.exp(-1j * wl * t)
    psi = w1 ** 2 * 0.2 * np.exp(-1j * w1 * t) + w2 ** 2 * 0.05j * np.exp(-1j * w2 * t) + wl ** 2 * low
    f_cut = 10 / T
    out = waveform.ffi_strain(psi, dt, f_cut)
    expect = h + low * (wl / (2 * math.pi * f_cut)) ** 2
    assert np.abs(out - expect).max() < 1e-12
