"""Psi4 extraction on the GPU (Sec. 2.3): modes l = 2..lmax against the
oracle on the same uploaded state (within 1e-9 of the largest mode: the two
sum the Ricci tensor, the interpolation and the quadrature in different
orders), for a linearised plane wave along a generic direction, a noisy
boosted and spinning puncture (every term of E and B active), both
precisions (the extraction reads the FP64 time level), evolved data, ragged
phi counts over the 128-thread rings, lmax up to 8; the closed form of the
plane wave's pinned case; argument errors."""

import pytest

import initial_data as idd
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

skbuild.build()


def _close(mg, mo, tol=1e-9):
    scale = max(abs(v) for v in mo.values())
    assert scale > 0
    for key in mo:
        assert abs(mg[key] - mo[key]) <= tol * scale, (key, mg[key], mo[key], scale)


def _grid(p, u, precision=0):
    g = sk.Grid(1, p.dx, [p], sk.Params(precision=precision), stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    return g


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nt,nph,lmax", [(16, 37, 4), (7, 130, 2), (20, 40, 8)])
def test_plane_wave_parity(precision, nt, nph, lmax):
    p = idd.centred_patch(40, 0.2)
    u = idd.plane_wave(p, 1e-6, 0.7e-6, 1.3, 1.1, 0.4)
    g = _grid(p, u, precision)
    c = (0.1, -0.05, 0.2)
    _close(g.psi4_modes(0, c, 2.5, nt, nph, lmax), oracle.psi4_modes(p, u, c, 2.5, nt, nph, lmax))


@pytest.mark.parametrize("precision", [0, 1])
def test_noisy_puncture_parity(precision):
    p = idd.centred_patch(40, 0.4)
    u = idd.bowen_york(p, 1.0, spin=(0.1, -0.2, 0.5), momentum=(0.1, 0.05, -0.1))
    u = idd.add_noise(p, u, 1e-5, idd.PUNCTURE_SEED)
    g = _grid(p, u, precision)
    _close(g.psi4_modes(0, (0.2, 0.1, -0.1), 5.0, 16, 32, 4), oracle.psi4_modes(p, u, (0.2, 0.1, -0.1), 5.0, 16, 32, 4))


def test_evolved_parity():
    p = idd.centred_patch(32, 0.5)
    u = idd.add_noise(p, idd.bowen_york(p, 1.0, spin=(0.0, 0.0, 0.4)), 1e-6, idd.PUNCTURE_SEED)
    g = _grid(p, u)
    for _ in range(3):
        g.rk4_step(0, 0.125)
    v = g.download_fields(0)
    _close(g.psi4_modes(0, (0.0, 0.0, 0.0), 5.0, 12, 24, 3), oracle.psi4_modes(p, v, (0.0, 0.0, 0.0), 5.0, 12, 24, 3))


def test_plane_wave_along_z_modes():
    """The case whose l = 2 modes the oracle pins against an independent
    quadrature of the closed form: the GPU gives the oracle's modes."""
    A, B, w, r = 1e-6, 0.4e-6, 1.2, 2.0
    p = idd.centred_patch(64, 0.125)
    u = idd.plane_wave(p, A, B, w, 0.0, 0.0)
    g = _grid(p, u)
    mg = g.psi4_modes(0, (0.0, 0.0, 0.0), r, 24, 48, 2)
    mo = oracle.psi4_modes(p, u, (0.0, 0.0, 0.0), r, 24, 48, 2)
    _close(mg, mo)
    assert abs(mg[(2, 2)]) > 1e-7


def test_errors():
    p = idd.centred_patch(32, 0.5)
    g = _grid(p, idd.minkowski(p))
    assert all(v == 0 for v in g.psi4_modes(0, (0.0, 0.0, 0.0), 5.0, 8, 16, 3).values())
    g.psi4_modes(0, (0.0, 0.0, 0.0), 7.5, 8, 16, 2)  # stencils reach the ghosts: accepted, as in the oracle
    for kw in [dict(radius=8.6), dict(lmax=1), dict(lmax=9), dict(ntheta=0), dict(nphi=0), dict(radius=-1.0),
               dict(ntheta=1024, nphi=1 << 20)]:
        args = dict(patch=0, centre=(0.0, 0.0, 0.0), radius=3.0, ntheta=8, nphi=16, lmax=2)
        args.update(kw)
        with pytest.raises(sk.SacrakError):
            g.psi4_modes(**args)
    assert all(v == 0 for v in g.psi4_modes(0, (0.0, 0.0, 0.0), 3.0, 8, 16, 2).values())
