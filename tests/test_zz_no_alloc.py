"""The allocation-free constraint monitor (sacrak_constraints_noalloc) against
the grid-based one (sacrak_constraints) and the CPU oracle, through the C ABI.

Callers that cannot allocate device memory (their device memory belongs to
another framework's pool, a fixed-size sandbox, a hook that must not call
cudaMalloc) pass a patch held in their own device memory; the partial sums
go to a fixed static device array shared by every call.  Two calls in a row
must both agree with the grid path and the oracle, which also shows that the
shared array keeps no state between calls that could leak into a result.
Invalid arguments are turned away before any launch: on the host by the
binding (wrong type, dtype, device, too few values) and in the library
(memory of another device, an allocation smaller than the patch array)."""
import ctypes

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


def _grid_norms(p, u, w_excise):
    g = sk.Grid(1, p.dx, [p], sk.Params())
    g.upload_fields(0, u)
    n = g.constraints(0, w_excise=w_excise)
    g.close()
    return n


def _cases():
    p1 = idd.single_puncture_patch(32, 8.0)
    p2 = idd.Patch(n=(40, 12, 20), dx=0.25, origin=(-5.0, -1.5, -2.5))
    u2 = idd.add_noise(p2, idd.punctures(p2, [0.6, 0.4], [(1.0, 0.1, 0.0), (-1.5, 0.0, 0.2)]), 1e-6, 3)
    return [(p1, idd.single_puncture_data(p1), 0.0), (p2, u2, 0.2)]


def test_noalloc_constraints_match_grid_path_and_oracle_twice():
    for p, u, wex in _cases():
        ref = _grid_norms(p, u, wex)
        _, orc = oracle.constraints(p, u, wex)
        dev = torch.as_tensor(u, device="cuda").contiguous()
        for _ in range(2):
            got = sk.constraints_noalloc(dev, p.n, p.dx, wex)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
            np.testing.assert_allclose(got, orc, rtol=1e-10, atol=0)
            assert np.all(got > 0)


def test_noalloc_rejects_sizes_beyond_limit():
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(dev, (513, 8, 8), 0.1)
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(np.zeros(8), (8, 8, 8), 0.1)  # host memory is not accepted


def test_noalloc_binding_rejects_bad_tensors_on_the_host():
    """Checked before the library is called: too few values, wrong dtype,
    not contiguous."""
    n = (8, 8, 8)
    need = 25 * 14 ** 3
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(torch.zeros(need - 1, dtype=torch.float64, device="cuda"), n, 0.1)
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(torch.zeros(need, dtype=torch.int64, device="cuda"), n, 0.1)
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(torch.zeros(2 * need, dtype=torch.float64, device="cuda")[::2], n, 0.1)


def _c_call(ptr, n, dx=0.1):
    out = np.empty(4)
    return sk.lib().sacrak_constraints_noalloc(ctypes.c_void_p(ptr), (ctypes.c_int * 3)(*n), dx, 0.0, None,
                                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def test_noalloc_library_rejects_a_short_allocation():
    """Called through the C ABI directly (no binding checks): a 500^3 patch
    array (26 GB) cannot fit the allocation of a small tensor, so the library
    returns SACRAK_EINVAL before any launch."""
    small = torch.zeros(1024, dtype=torch.float64, device="cuda")
    assert _c_call(small.data_ptr(), (500, 500, 500)) == sk.EINVAL
    # the library still works afterwards
    p, u, wex = _cases()[0]
    ref = _grid_norms(p, u, wex)
    np.testing.assert_allclose(sk.constraints_noalloc(torch.as_tensor(u, device="cuda"), p.n, p.dx, wex), ref,
                               rtol=1e-12)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second CUDA device")
def test_noalloc_library_rejects_memory_of_another_device():
    """Memory of device 1 while device 0 is current: SACRAK_EINVAL from the
    pointer check, no kernel launched."""
    torch.cuda.set_device(0)
    other = torch.zeros(25 * 14 ** 3, dtype=torch.float64, device="cuda:1")
    assert _c_call(other.data_ptr(), (8, 8, 8)) == sk.EINVAL
    with pytest.raises(sk.SacrakError):
        sk.constraints_noalloc(other, (8, 8, 8), 0.1)
