"""The grid checkerboard of Minkowski space through the C ABI (both
precisions) against the hand-derived linear RK4 map of
tests/test_oracle_courant.py: the stage kernels carry the same discrete
operator as the oracle, so the paper's Courant factor is past the linear
limit on the GPU as well (Sec. 2.2)."""
import numpy as np
import pytest

import initial_data as idd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2607_08743_gb300 as sk
from paper_2607_08743_gb300 import build as skbuild

from tests.test_oracle_courant import ALP, _amplitudes, _checkerboard, _operator, _rk4_map

skbuild.build()


@pytest.mark.parametrize("precision,courant,khat", [(0, 0.5, 0), (0, 0.5, 1), (0, 0.25, 0), (1, 0.5, 0),
                                                    (1, 0.25, 1)])
def test_checkerboard_mode_on_the_gpu(precision, courant, khat):
    n, eps = 16, 1e-9
    p = idd.centred_patch(n, 1.0 / n)
    cb = _checkerboard(p)
    u = idd.minkowski(p)
    u[ALP] += eps * cb
    g = sk.Grid(1, p.dx, [p], sk.Params(bc=1, courant=courant, precision=precision, lapse_uses_khat=khat),
                stream=torch.cuda.Stream())
    g.upload_fields(0, u)
    dt = courant * p.dx
    M = _rk4_map(dt * _operator(p.dx, khat, 0.5, 0.005))
    y = np.array([eps, 0.0, 0.0, 0.0])
    # FP64: rounding of O(1) fields; mixed: FP32 arithmetic on FP64-formed
    # differences, 2^-24 of the mode per step
    tol = 1e-7 if precision == 0 else 3e-6
    for _ in range(5):
        g.rk4_step(0, dt)
        y = M @ y
    got = _amplitudes(p, g.download_fields(0), cb)
    g.close()
    np.testing.assert_allclose(got, y, rtol=0, atol=tol * np.abs(y).max() + 1e-13)
    assert (np.abs(y).max() > 100 * eps) == (courant == 0.5 and khat == 0)
