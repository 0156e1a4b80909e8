"""Grouped transforms of host-resident channels streamed through the GPU in
chunks (dsbt_*_grouped_host): results equal the device entry points on the
same inputs, for chunk cuts inside and between l groups, pinned and pageable
host memory, both precisions."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1509_07115_gb300 import dsbt, inputs


def test_host_entry_points_reject_bad_arguments():
    lib = dsbt.load()
    counts = (ctypes.c_int * 3)(1, 1, 1)
    assert lib.dsbt_host_workspace_size(None, counts, 4, 8) == 0
    assert lib.dsbt_kinetic_grouped_host(None, counts, 4, 0.1, None, None, 8, None, 0, None) == -1
    assert lib.dsbt_forward_grouped_host(None, counts, 4, None, None, 8, None, 0, None) == -1
    assert lib.dsbt_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("chunks", [1, 3, 8, 1000])
def test_kinetic_host_equals_device(lib, chunks):
    N, lmax = 1024, 12
    counts = [2 * l + 1 for l in range(lmax + 1)]
    counts[4] = 0
    p = lib.Plan(N, 0.1 * N, lmax, fp64=False)
    x = inputs.gaussian_sum(31, N, 0.1, counts).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    ref = p.kinetic_grouped(counts, xd, 0.05).cpu()
    xh = torch.from_numpy(x).pin_memory()
    yh = p.kinetic_grouped_host(counts, xh, 0.05, chunks=chunks)
    torch.cuda.synchronize()
    assert torch.equal(yh, ref)
    p.close()


@pytest.mark.gpu
def test_forward_inverse_host_fp64_and_pageable(lib):
    N, lmax = 768, 7
    counts = [3] * (lmax + 1)
    p = lib.Plan(N, 0.1 * N, lmax, tf32x3=False)
    x = inputs.gaussian_sum(32, N, 0.1, counts)
    xd = torch.from_numpy(x).cuda()
    b_ref = p.forward_grouped(counts, xd).cpu()
    xh = torch.from_numpy(x)                         # pageable
    bh = p.forward_grouped_host(counts, xh, chunks=5)
    torch.cuda.synchronize()
    assert torch.equal(bh, b_ref)
    y_ref = p.inverse_grouped(counts, b_ref.cuda()).cpu()
    yh = p.inverse_grouped_host(counts, bh.pin_memory(), chunks=2)
    torch.cuda.synchronize()
    assert torch.equal(yh, y_ref)
    p.close()
