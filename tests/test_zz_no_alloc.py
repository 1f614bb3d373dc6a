"""The allocation-free constraint monitor (sacrak_constraints_noalloc) against
the grid-based one (sacrak_constraints), through the C ABI.

Callers that cannot allocate device memory (their device memory belongs to
another framework's pool, a fixed-size sandbox, a hook that must not call
cudaMalloc) pass a patch held in their own device memory; the partial sums
go to a fixed static device array shared by every call.  Two calls in a row
must both agree with the grid path, which also shows that the shared array
keeps no state between calls that could leak into a result."""
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


def _grid_norms(p, u, w_excise):
    g = sk.Grid(1, p.dx, [p], sk.Params())
    g.upload_fields(0, u)
    n = g.constraints(0, w_excise=w_excise)
    g.close()
    return n


def test_noalloc_constraints_match_grid_path_twice():
    cases = []
    p1 = idd.single_puncture_patch(32, 8.0)
    cases.append((p1, idd.single_puncture_data(p1), 0.0))
    p2 = idd.Patch(n=(40, 12, 20), dx=0.25, origin=(-5.0, -1.5, -2.5))
    u2 = idd.add_noise(p2, idd.punctures(p2, [0.6, 0.4], [(1.0, 0.1, 0.0), (-1.5, 0.0, 0.2)]), 1e-6, 3)
    cases.append((p2, u2, 0.2))
    for p, u, wex in cases:
        ref = _grid_norms(p, u, wex)
        dev = torch.as_tensor(u, device="cuda").contiguous()
        for _ in range(2):
            got = sk.constraints_noalloc(dev, p.n, p.dx, wex)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
            assert np.all(got > 0)


def test_noalloc_rejects_sizes_beyond_limit():
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(dev, (513, 8, 8), 0.1)
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(np.zeros(8), (8, 8, 8), 0.1)  # host memory is not accepted
