"""Properties of the analytic inputs that the diagnostics' pins rely on
(no GPU): Bowen-York extrinsic curvature trace-free and divergence-free in
the flat conformal metric (the momentum constraint away from the puncture),
and the linearised plane wave transverse and traceless with unit determinant
of the conformal metric."""
import numpy as np

import initial_data as idd


def _ahat(p, u):
    """psi^6 At = Ahat (W^3 = psi^-6) as a 3 x 3 field."""
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    A = np.zeros((3, 3) + u.shape[1:])
    for a, (i, j) in enumerate(sym):
        A[i, j] = A[j, i] = u[9 + a] / u[0] ** 3
    return A


def _by_divergence(n):
    p = idd.centred_patch(n, 12.0 / n)
    u = idd.bowen_york(p, 1.0, centre=(0.3, -0.2, 0.1), spin=(0.2, -0.1, 0.5), momentum=(0.1, 0.3, -0.2))
    A = _ahat(p, u)
    h = p.dx

    def d(f, axis):  # 4th-order centred difference; array axes (z, y, x)
        return (8 * (np.roll(f, -1, axis) - np.roll(f, 1, axis)) - (np.roll(f, -2, axis) - np.roll(f, 2, axis))) / (12 * h)
    z, y, x = np.meshgrid(p.axis(2), p.axis(1), p.axis(0), indexing="ij")
    r = np.sqrt((x - 0.3) ** 2 + (y + 0.2) ** 2 + (z - 0.1) ** 2)
    mask = (r > 2.0) & (np.abs(x) < 5) & (np.abs(y) < 5) & (np.abs(z) < 5)
    tr = np.abs(A[0, 0] + A[1, 1] + A[2, 2]).max() / np.abs(A).max()
    div = max(np.abs(d(A[i, 0], 2) + d(A[i, 1], 1) + d(A[i, 2], 0))[mask].max() for i in range(3))
    return tr, div


def test_bowen_york_trace_and_divergence_free():
    tr1, d1 = _by_divergence(48)
    tr2, d2 = _by_divergence(96)
    assert tr1 < 1e-12 and tr2 < 1e-12
    assert d1 / d2 > 10, (d1, d2)  # a truncation error of 4th order, not a non-zero divergence


def test_plane_wave_transverse_traceless():
    p = idd.centred_patch(16, 0.5)
    for th, ph in ((0.0, 0.0), (1.1, 0.4), (2.3, -2.0)):
        k, e1, e2 = idd.plane_wave_basis(th, ph)
        assert abs(np.dot(k, e1)) < 1e-15 and abs(np.dot(k, e2)) < 1e-15 and abs(np.dot(e1, e2)) < 1e-15
        u = idd.plane_wave(p, 1e-6, 0.5e-6, 1.0, th, ph)
        sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        g = np.zeros((3, 3) + u.shape[1:])
        for a, (i, j) in enumerate(sym):
            g[i, j] = g[j, i] = u[1 + a]
        det = np.linalg.det(np.moveaxis(g, (0, 1), (-2, -1)))
        assert np.abs(det - 1.0).max() < 1e-13
        h = g - np.eye(3)[:, :, None, None, None]
        # transverse (k.h = 0) and traceless to first order in the amplitude
        assert np.abs(np.einsum("i,ij...->j...", k, h)).max() < 1e-11
        assert np.abs(h[0, 0] + h[1, 1] + h[2, 2]).max() < 1e-11
