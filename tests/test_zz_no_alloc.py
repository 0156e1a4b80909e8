"""dsbt_forward_grouped_noalloc: the grouped forward for callers that cannot
allocate device memory (framework-owned device memory, loops that cannot take
cudaMalloc's implicit synchronisation, fixed memory budgets).  It must give the
results of dsbt_forward_grouped, which takes a caller workspace, on repeated
calls (the static scratch keeps the previous call's contents), for every kind
of plan (the dense factors, and the interval schemes of DSBT_PLAN_FAST64 and
DSBT_PLAN_FAST_SPLIT, whose extra scratch also lives in the static array), and
reject requests larger than its 64 MiB scratch before launching anything.

Collected last (file name) so that a stop-at-first-failure run has already run
every other test when this one runs.
"""
import ctypes

import pytest
import torch

from paper_1509_07115_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 1e-6}
PLANS = {"dense": {}, "fast64": {"fast64": True}, "fast_split": {"fast_split": True}}


@pytest.mark.parametrize("kind", sorted(PLANS))
def test_noalloc_forward_matches_workspace_forward(lib, kind):
    so = lib.load()
    so.dsbt_forward_grouped_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    N, lmax = 1024, 9
    plan = lib.Plan(N, 102.4, lmax, fp64=True, tf32x3=True, **PLANS[kind])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for dtype in (torch.complex128, torch.complex64):
        for seed, counts in ((3, [2 * l + 1 for l in range(lmax + 1)]), (4, [3, 0, 1, 7, 0, 2, 1, 0, 5, 4])):
            x = inputs.gaussian_sum(seed, N, 0.1, counts, dtype=dtype, device="cuda")
            ref = plan.forward_grouped(counts, x)
            arr = (ctypes.c_int * len(counts))(*counts)
            nrm = torch.linalg.vector_norm(x.to(torch.complex128), dim=1)
            for _ in range(2):   # two calls in a row on the shared scratch
                out = torch.full_like(x, float("nan"))
                rc = so.dsbt_forward_grouped_noalloc(plan.handle, arr, lib.DTYPES[dtype],
                                                     ctypes.c_void_p(x.data_ptr()),
                                                     ctypes.c_void_p(out.data_ptr()), stream)
                assert rc == 0, so.dsbt_last_error()
                torch.cuda.synchronize()
                err = ((out - ref).abs().amax(dim=1).to(torch.float64) / nrm).max().item()
                assert err < TOL[dtype], (kind, dtype, err)
    # a request beyond the 64 MiB scratch is refused on the host
    big = [0] * (lmax + 1)
    big[0] = 1 << 13
    arr = (ctypes.c_int * len(big))(*big)
    dummy = torch.empty(1, dtype=torch.complex64, device="cuda")
    rc = so.dsbt_forward_grouped_noalloc(plan.handle, arr, lib.DTYPES[torch.complex64],
                                         ctypes.c_void_p(dummy.data_ptr()),
                                         ctypes.c_void_p(dummy.data_ptr() + 8), stream)
    assert rc == -1 and b"64" in so.dsbt_last_error()
    assert plan.device_status() == 0
    plan.close()
