"""Failure paths of the C ABI on the GPU, made without faulting anything:

* a non-finite value in uploaded data makes the next stage kernel set the
  device error flag; the next synchronising call returns SACRAK_ENONFINITE,
  stepping calls then return SACRAK_ESTATE, and new data make the grid
  usable again (both precisions);
* the TMA stage kernels' bounded wait for a field's copy: with the test hook
  that makes every wait count as run out, the kernel stops issuing copies,
  lets the copies in flight land, returns without writing, and the next
  synchronising call returns SACRAK_ETIMEOUT; the grid recovers with the
  default bound and new data."""
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


def _expect_status(status, fn, *a):
    with pytest.raises(sk.SacrakError) as e:
        fn(*a)
    assert e.value.status == status, e.value


def _step_then_sync(g):
    """rk4_step does not synchronise; the download after it does."""
    g.rk4_step(0)
    g.download_fields(0)


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_upload_is_reported_and_recovered(precision):
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    g = sk.Grid(1, p.dx, [p], sk.Params(precision=precision))
    bad = u.copy()
    bad[7, 12, 15, 20] = np.nan  # Khat at one active point
    g.upload_fields(0, bad)
    _expect_status(sk.ENONFINITE, _step_then_sync, g)
    _expect_status(sk.ESTATE, g.rk4_step, 0)      # invalid until new data
    g.upload_fields(0, u)
    dt = 0.5 * p.dx
    g.rk4_step(0, dt)
    got = g.download_fields(0)
    assert np.all(np.isfinite(got))
    ref = oracle.rk4_step(p, u, dt, oracle.Params())
    a = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    ch = np.abs(ref[a] - u[a]).max(axis=(1, 2, 3))
    err = (np.abs(got[a] - ref[a]).max(axis=(1, 2, 3)) / np.where(ch > 0, ch, 1.0)).max()
    assert err <= (1e-4 if precision else 1e-9), err
    g.close()


@pytest.mark.parametrize("kernel", [1, 3])
def test_tma_wait_timeout_is_reported_and_recovered(kernel):
    p = idd.single_puncture_patch(32, 8.0)
    u = idd.single_puncture_data(p)
    g = sk.Grid(1, p.dx, [p], sk.Params(precision=1))
    g.set_stage_kernel(0, kernel)
    g.upload_fields(0, u)
    g.set_wait_limit(-1)
    _expect_status(sk.ETIMEOUT, _step_then_sync, g)
    _expect_status(sk.ESTATE, g.rk4_step, 0)
    g.set_wait_limit(0)
    g.upload_fields(0, u)
    dt = 0.5 * p.dx
    g.rk4_step(0, dt)
    got = g.download_fields(0)
    ref = oracle.rk4_step(p, u, dt, oracle.Params())
    a = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    ch = np.abs(ref[a] - u[a]).max(axis=(1, 2, 3))
    err = (np.abs(got[a] - ref[a]).max(axis=(1, 2, 3)) / np.where(ch > 0, ch, 1.0)).max()
    assert err <= 1e-4, err
    # the captured coarse step picks the bound up as well
    g.set_wait_limit(-1)
    _expect_status(sk.ETIMEOUT, lambda: (g.level_step(0), g.constraints(0)))
    g.close()
