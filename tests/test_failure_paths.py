"""Failure detection without a GPU fault.

* A corrupt factor is injected on the host (dsbt_plan_perturb_T adds a small
  error to one entry of the FP64 T_l); the orthogonality probe of Eq. (25)
  (T^T T = I) then fails with DSBT_ERR_PLAN_CHECK, and passes again once the
  entry is restored.
* A device-side wait is made to run out: with a spin limit of one poll every
  bounded mbarrier wait of the tensor-core kernels that is not already
  satisfied gives up at once.  The kernel lets its own TMA copies and MMAs
  finish, frees its TMEM and returns; the host reads the timeout from the
  plan's status word, and the next call with the default limit (and a call on
  a fresh plan) gives the right result: the context stays usable.
No kernel is made to trap, hang or touch a bad address.
"""
import ctypes

import pytest
import torch

from paper_1509_07115_gb300 import dsbt, inputs


def test_hooks_reject_null_plan_on_host():
    lib = dsbt.load()
    assert lib.dsbt_plan_check(None, None, None) == -1
    assert lib.dsbt_plan_set_spin_limit(None, 1) == -1
    assert lib.dsbt_plan_perturb_T(None, 0, 0, 0, 1.0, None) == -1
    assert lib.dsbt_plan_set_fast_lag(None, 1) == -1


@pytest.mark.gpu
def test_corrupt_factor_fails_the_plan_check(lib):
    p = lib.Plan(256, 25.6, 8, tf32x3=False)
    assert p.check() < 1e-13
    p.perturb_T(5, 100, 50, 1e-6)
    with pytest.raises(lib.DSBTError) as ei:
        p.check()
    assert "(-3)" in str(ei.value)
    p.perturb_T(5, 100, 50, -1e-6)
    assert p.check() < 1e-13
    p.close()


@pytest.mark.gpu
@pytest.mark.parametrize("fast", [False, True])
def test_device_wait_timeout_is_reported_and_recovered(lib, fast):
    N, lmax = 1024, 9
    counts = [2 * l + 1 for l in range(lmax + 1)]
    x = inputs.gaussian_sum(31, N, 0.1, counts, dtype=torch.complex64, device="cuda")
    p = lib.Plan(N, 0.1 * N, lmax, fp64=False, tf32x3=True, fast_split=fast)
    ref = p.forward_grouped(counts, x)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    p.set_spin_limit(1)
    p.forward_grouped(counts, x)                  # results undefined: the waits gave up
    torch.cuda.synchronize()
    assert p.device_status(reset=True) == 1
    p.set_spin_limit(0)                           # default limit
    again = p.forward_grouped(counts, x)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert torch.equal(again, ref)
    p.close()
    fresh = lib.Plan(N, 0.1 * N, lmax, fp64=False, tf32x3=True, fast_split=fast)
    assert torch.equal(fresh.forward_grouped(counts, x), ref)
    assert fresh.device_status() == 0
    fresh.close()
