"""The refined levels' ghost fills and prolongations on the library's second
stream, beside the stage kernels (sacrak_set_overlap, the default), give
the same results bit for bit as every launch on the grid's stream in order:
captured coarse steps and eager ones, both precisions, equatorial symmetry,
tracked and moved patches, a single refined-level RK4 step (Sec. 2.2.1)."""
import numpy as np
import pytest

import initial_data as idd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

skbuild.build()


def _pair(h, states, stream_kind, **prm):
    grids = []
    for on in (True, False):
        st = torch.cuda.Stream() if stream_kind == "graph" else torch.cuda.default_stream()
        g = sk.Grid(len(h.levels), h.dx0, h.patches, sk.Params(**prm), stream=st)
        g.set_overlap(on)
        for i, u in enumerate(states):
            g.upload_fields(i, u)
        grids.append(g)
    return grids


def _same(a, b, npatch):
    for i in range(npatch):
        x, y = a.download_fields(i), b.download_fields(i)
        assert np.array_equal(x, y), (i, np.abs(x - y).max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("stream_kind", ["graph", "eager"])
def test_overlap_bitwise_binary(precision, stream_kind):
    h = idd.small_binary()
    states = idd.hierarchy_data(h, noise=1e-10)
    a, b = _pair(h, states, stream_kind, precision=precision)
    for _ in range(3):
        a.level_step(0)
        b.level_step(0)
    _same(a, b, len(h.patches))
    # a single RK4 step of the finest level, then a coarse step again
    lf = len(h.levels) - 1
    a.rk4_step(lf)
    b.rk4_step(lf)
    _same(a, b, len(h.patches))
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_overlap_bitwise_zsym(precision):
    h = idd.small_binary(n_fixed=24, n_moving=16, n_levels=3, n_fixed_levels=2, dx0=1.0, sep=2.0)
    hh = idd.upper_half_hierarchy(h)
    half = [idd.upper_half_array(p, u) for p, u in zip(h.patches, idd.hierarchy_data(h, noise=0.0))]
    a, b = _pair(hh, half, "graph", precision=precision, zsym=1)
    for _ in range(2):
        a.level_step(0)
        b.level_step(0)
    _same(a, b, len(hh.patches))


def test_overlap_bitwise_moving_patches():
    h = idd.moving_binary_3_level()
    states = idd.hierarchy_data(h, noise=1e-8)
    for u in states:
        u[19] += 0.3
    a, b = _pair(h, states, "graph", precision=1)
    follow = [-1, 0, 1, 0, 1]
    for g in (a, b):
        g.track_punctures(h.positions, follow)
    for step in range(3):
        for g in (a, b):
            g.level_step(0)
            if step == 1:
                g.move_patch(3, (1, 0, 0))
    _same(a, b, len(h.patches))
    assert np.array_equal(a.punctures(), b.punctures())


def test_overlap_argument_checked():
    p = idd.centred_patch(8, 1.0)
    g = sk.Grid(1, p.dx, [p], sk.Params())
    with pytest.raises(sk.SacrakError):
        lib = sk.lib()
        g._check(lib.sacrak_set_overlap(g._h, 2), "set_overlap")
    g.close()
