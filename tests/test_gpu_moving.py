"""Moving boxes on the GPU (Sec. 2.2.1): puncture tracking dx/dt = -beta
inside the captured coarse step, explicit patch shifts and the regrid rule,
against the oracle's BOHierarchy doing the same.  FP64: states 1e-12 right
after a shift and 1e-10 after further coarse steps, puncture positions 1e-12;
mixed precision: the shift itself is FP64 (1e-12), evolved states 1e-4 of
the step's change, positions 1e-8.  Also the argument and state errors."""
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
from tests.gpu_common import rel_err

skbuild.build()

FOLLOW = [-1, 0, 1, 0, 1]


def _setup(precision, shift=(0.0, 0.0, 0.0), noise=1e-8):
    h = idd.moving_binary_3_level()
    states = idd.hierarchy_data(h, noise=noise)
    for u in states:
        for d in range(3):
            u[19 + d] += shift[d]
    g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(precision=precision, courant=0.5),
                stream=torch.cuda.Stream())
    for i, u in enumerate(states):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    return h, states, g, bo


def _change_err(v, vo, u0, g=3):
    a = (slice(None), slice(g, -g), slice(g, -g), slice(g, -g))
    d = np.abs(v[a] - vo[a]).max(axis=(1, 2, 3))
    s = np.abs(vo[a] - u0[a]).max(axis=(1, 2, 3))
    return np.where(s > 0, d / np.where(s > 0, s, 1.0), d)


def _compare(g, bo, precision, ref_states, tol64, active_only=True):
    for i in range(len(bo.patches)):
        v = g.download_fields(i)
        if precision == 0:
            e = rel_err(v, bo.current(i), active_only=active_only)
        else:
            e = _change_err(v, bo.current(i), ref_states[i])
        assert e.max() <= (tol64 if precision == 0 else 1e-4), (i, dict(zip(idd.FIELD_NAMES, e)))


def _replay(h, g):
    """An oracle hierarchy holding the GPU's current states (the shift itself
    is then compared on identical inputs in both precisions)."""
    return oracle.BOHierarchy(h, [g.download_fields(i) for i in range(len(h.patches))], oracle.Params(),
                              courant=0.5)


MOVES = {
    "l1+l2": ((1, (-1, 1, 0)), (4, (1, -1, 2))),  # a level-1 patch with its child, then a level-2 patch
    "l2": ((3, (1, 0, 0)),),                     # a level-2 patch under a level with full history
    "l2z": ((4, (0, 0, -1)), (3, (-1, 2, 0))),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("moves", sorted(MOVES))
def test_move_patch_parity(precision, moves):
    h, states, g, bo = _setup(precision)
    g.level_step(0)
    bo.level_step(0)
    before = [bo.current(i).copy() for i in range(5)]
    rep = _replay(h, g)
    for pid, s in MOVES[moves]:
        g.move_patch(pid, s)
        bo.move_patch(pid, s)
        rep.move_patch(pid, s)
    # the shifted data themselves (FP64 on both sides, ghosts included)
    for i in range(5):
        assert rel_err(g.download_fields(i), rep.current(i)).max() <= 1e-12, i
    for _ in range(2):
        g.level_step(0)
        bo.level_step(0)
    _compare(g, bo, precision, before, 1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_tracking_parity(precision):
    h, states, g, bo = _setup(precision, shift=(0.3, -0.1, 0.05))
    g.track_punctures(h.positions, FOLLOW)
    bo.track(h.positions, FOLLOW)
    for _ in range(3):
        g.level_step(0)
        bo.level_step(0)
    pg = g.punctures()
    po = np.array(bo.punct)
    tol = 1e-12 if precision == 0 else 1e-8
    assert np.abs(pg - po).max() <= tol, (pg, po)
    # the punctures moved against the shift
    assert pg[0][0] < h.positions[0][0] - 0.1


@pytest.mark.parametrize("precision", [0, 1])
def test_regrid_parity(precision):
    h, states, g, bo = _setup(precision)
    g.track_punctures(h.positions, FOLLOW)
    bo.track(h.positions, FOLLOW)
    g.level_step(0)
    bo.level_step(0)
    before = [bo.current(i).copy() for i in range(5)]
    # displace the punctures (as after a long run) and regrid both
    moved_pos = [(1.9, 0.6, 0.0), (-3.0, -1.55, 0.3)]
    rep = _replay(h, g)
    for x in (g, rep, bo):
        (x.track_punctures if x is g else x.track)(moved_pos, FOLLOW)
    mg = g.regrid()
    assert mg == rep.regrid() == bo.regrid() and mg >= 3
    for i in range(5):
        assert rel_err(g.download_fields(i), rep.current(i)).max() <= 1e-12, i
        assert g.patch_origin(i) == pytest.approx(rep.patches[i].origin, abs=0.0)
    assert g.regrid() == 0  # nothing left to do
    for _ in range(2):
        g.level_step(0)
        bo.level_step(0)
    _compare(g, bo, precision, before, 1e-10)
    if precision == 0:
        assert np.abs(g.punctures() - np.array(bo.punct)).max() <= 1e-12


def test_errors():
    h, states, g, bo = _setup(0)
    with pytest.raises(sk.SacrakError):
        g.move_patch(0, (1, 0, 0))  # level 0
    with pytest.raises(sk.SacrakError):
        g.move_patch(3, (5, 0, 0))  # child would leave its parent's margin
    with pytest.raises(sk.SacrakError):
        g.move_patch(1, (0, 3, 0))  # would push its child out of the margin
    with pytest.raises(sk.SacrakError):
        g.track_punctures(h.positions, [-1, 0, 2, 0, 1])  # puncture 2 does not exist
    with pytest.raises(sk.SacrakError):
        g.track_punctures(h.positions, [-1, 0, 0, 0, -1])  # puncture 1 followed by no patch
    with pytest.raises(sk.SacrakError):
        g.track_punctures(h.positions, [0, 0, 1, 0, 1])  # level 0 cannot follow
    with pytest.raises(sk.SacrakError):
        g.track_punctures([(0.0, 0.0, 0.0)] * 9, [-1, 0, 1, 0, 1])
    # not between coarse steps: one step of level 1 alone
    g.level_step(1)
    with pytest.raises(sk.SacrakError):
        g.move_patch(3, (1, 0, 0))
    # a tracking stencil outside its patch: reported once, the grid stays usable
    h, states, g, bo = _setup(0)
    g.track_punctures([(9.0, 0.0, 0.0), (-3.0, 0.0, 0.0)], FOLLOW)
    g.level_step(0)
    with pytest.raises(sk.SacrakError):
        g.punctures()
    assert np.allclose(g.punctures()[0], (9.0, 0.0, 0.0))
    g.track_punctures(h.positions, FOLLOW)
    g.level_step(0)
    assert np.all(np.isfinite(g.punctures()))


def test_half_domain_shift_parity():
    """Equatorial symmetry with patch shifts: the GPU's half-domain grid
    against the oracle's half-domain hierarchy doing the same shifts."""
    h = idd.moving_binary_3_level()
    states = idd.hierarchy_data(h, noise=0.0)
    for u in states:
        u[19] += 0.2
        u[20] -= 0.1
    hh = idd.upper_half_hierarchy(h)
    half = [idd.upper_half_array(p, u) for p, u in zip(h.patches, states)]
    g = sk.Grid(len(hh.levels), hh.dx0, hh.patches, sk.Params(courant=0.5, zsym=1), stream=torch.cuda.Stream())
    for i, u in enumerate(half):
        g.upload_fields(i, u)
    bo = oracle.BOHierarchy(hh, half, oracle.Params(), courant=0.5, zsym=True)
    for x in (g, bo):
        x.level_step(0)
        x.move_patch(1, (-1, 1, 0))
        x.move_patch(4, (1, 0, 0))
        x.level_step(0)
    with pytest.raises(sk.SacrakError):
        g.move_patch(3, (0, 0, 1))
    for i in range(len(hh.patches)):
        assert rel_err(g.download_fields(i), bo.current(i), active_only=True).max() <= 1e-10, i
