"""ADM mass, angular momentum (Sec. 2.3) and linear momentum (Sec. 3.2)
surface integrals on the GPU:
parity with the oracle on the same uploaded state (relative 1e-11: the two
sum the same terms in different orders), on data where every term of both
integrands is active (noise on all fields), spheres whose phi points leave a
ragged tail over the 128-thread rings, a refined patch away from the origin,
both precisions (the integrals read the FP64 time level), after evolution,
and the argument and patch-edge errors."""
import numpy as np
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

TOL = 1e-11


def _close(a, b, scale):
    return abs(a - b) <= TOL * max(1.0, abs(scale))


def _all_close(vg, vo):
    """M relative to itself, J_z and P relative to the largest of them and M."""
    s = max(abs(v) for v in vo)
    return _close(vg[0], vo[0], vo[0]) and all(_close(a, b, s) for a, b in zip(vg[1:], vo[1:]))


def _noisy_spin(p, amp=1e-3, centre=(0.0, 0.0, 0.0)):
    u = idd.bowen_york(p, 1.0, centre, spin=(0.1, -0.2, 0.6), momentum=(0.05, 0.1, -0.03))
    return idd.add_noise(p, u, amp, idd.PUNCTURE_SEED)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nt,nph", [(24, 48), (17, 300), (1, 1), (64, 129)])
def test_parity_uniform(precision, nt, nph):
    p = idd.centred_patch(40, 0.4)
    u = _noisy_spin(p)
    g = sk.Grid(1, p.dx, [p], sk.Params(precision=precision), stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    c = (0.3, -0.1, 0.2)
    for r in (2.0, 5.5):
        vg = g.adm_integrals(0, c, r, nt, nph)
        vo = oracle.adm_integrals(p, u, c, r, nt, nph)
        assert _all_close(vg, vo), (r, vg, vo)


def test_closed_forms_on_gpu():
    """Schwarzschild M (1 + M/(2r)), Bowen-York J_z = S_z and P^ADM = P
    straight from the GPU, within the oracle-pinned discretisation error."""
    p = idd.centred_patch(64, 0.25)
    u = idd.bowen_york(p, 1.0, spin=(0.0, 0.0, 0.7), momentum=(0.1, -0.2, 0.05))
    g = sk.Grid(1, p.dx, [p], sk.Params(), stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    for r in (4.5, 6.0):
        m, j, *P = g.adm_integrals(0, (0.0, 0.0, 0.0), r, 48, 96)
        assert abs(m - (1.0 + 1.0 / (2.0 * r))) < 1e-3 * p.dx ** 4
        assert abs(j - 0.7) < 2e-6
        assert max(abs(a - b) for a, b in zip(P, (0.1, -0.2, 0.05))) < 5e-6


def test_pi_symmetric_momentum_vanishes():
    """pi-symmetric data (Sec. 3.2): P_x and P_y vanish to rounding on a
    sphere centred on the rotation axis, while P_z of the same data does not
    (momentum along z is pi-symmetric)."""
    p = idd.centred_patch(40, 0.4)
    u = idd.add_noise(p, idd.bowen_york(p, 1.0, momentum=(0.0, 0.0, 0.2)), 1e-4, idd.PUNCTURE_SEED)
    u = idd.symmetrise_pi(p, u)
    g = sk.Grid(1, p.dx, [p], sk.Params(), stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    assert g.pi_symmetry(0) == 0.0
    m, j, px, py, pz = g.adm_integrals(0, (0.0, 0.0, 0.0), 5.0, 24, 48)
    assert abs(px) < 1e-15 and abs(py) < 1e-15
    assert abs(pz - 0.2) < 1e-3


def test_parity_refined_patch():
    """A level-1 patch away from the origin in a 2-level grid."""
    h = idd.small_binary(n_fixed=24, n_moving=16, n_levels=2, n_fixed_levels=1)
    states = idd.hierarchy_data(h, noise=1e-4)
    pats = h.patches
    g = sk.Grid(len(h.levels), h.dx0, pats, sk.Params(), stream=torch.cuda.Stream())
    for i, (pp, uu) in enumerate(zip(pats, states)):
        g.upload_fields(i, uu)
    for i, pp in enumerate(pats):
        if pp.level == 0:
            continue
        c = tuple(pp.origin[d] + 0.5 * pp.n[d] * pp.dx + 0.13 * pp.dx for d in range(3))
        r = 0.5 * min(pp.n) * pp.dx - 5.5 * pp.dx
        vg = g.adm_integrals(i, c, r, 20, 40)
        vo = oracle.adm_integrals(pp, states[i], c, r, 20, 40)
        assert _all_close(vg, vo), (i, vg, vo)


@pytest.mark.parametrize("precision", [0, 1])
def test_parity_after_evolution(precision):
    p = idd.centred_patch(32, 0.5)
    u = _noisy_spin(p, amp=1e-6)
    g = sk.Grid(1, p.dx, [p], sk.Params(precision=precision), stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    for _ in range(3):
        g.rk4_step(0, 0.25 * p.dx)
    v = g.download_fields(0)
    vg = g.adm_integrals(0, (0.0, 0.0, 0.0), 5.0, 24, 48)
    vo = oracle.adm_integrals(p, v, (0.0, 0.0, 0.0), 5.0, 24, 48)
    assert _all_close(vg, vo), (vg, vo)


def test_errors():
    p = idd.centred_patch(32, 0.5)
    g = sk.Grid(1, p.dx, [p], sk.Params(), stream=torch.cuda.Stream())
    g.upload_fields(0, idd.minkowski(p))
    assert g.adm_integrals(0, (0.0, 0.0, 0.0), 5.0, 8, 16) == (0.0,) * 5
    # the oracle accepts r = 7.5 on this patch (its stencils reach the ghosts)
    # and rejects r = 8.6; the GPU draws the same line
    g.adm_integrals(0, (0.0, 0.0, 0.0), 7.5, 8, 16)
    with pytest.raises(sk.SacrakError):
        g.adm_integrals(0, (0.0, 0.0, 0.0), 8.6, 8, 16)
    for bad in [dict(radius=0.0), dict(radius=-1.0), dict(ntheta=0), dict(ntheta=1025), dict(nphi=0),
                dict(radius=float("nan"))]:
        kw = dict(patch=0, centre=(0.0, 0.0, 0.0), radius=2.0, ntheta=8, nphi=16)
        kw.update(bad)
        with pytest.raises(sk.SacrakError):
            g.adm_integrals(**kw)
    with pytest.raises(sk.SacrakError):
        g.adm_integrals(1, (0.0, 0.0, 0.0), 2.0, 8, 16)
    # the grid stays usable after a rejected call
    assert g.adm_integrals(0, (0.0, 0.0, 0.0), 3.0, 8, 16) == (0.0,) * 5
