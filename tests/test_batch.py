"""Batch of uneven transforms (different N_t and l_max_t) with one shared factor
set: every transform against the oracle built at its own N (which checks that
the regular rows of T_l do not depend on N and that the per-N completion rows
are right), the kinetic step against the single-plan path, and CUDA-graph
replay against the direct call."""
import numpy as np
import pytest
import torch

import oracle
from paper_1509_07115_gb300 import inputs

pytestmark = pytest.mark.gpu

TRANSFORMS = [(256, 3), (768, 9), (512, 6), (1280, 12), (256, 20), (1024, 2)]
DR = 0.1


def make(lib):
    trs = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in TRANSFORMS]
    trs[1][2][4] = 0          # an empty group
    b = lib.Batch(trs, DR, autotune=True)
    xs = [inputs.gaussian_sum(20 + k, N, DR, c).astype(np.complex64) for k, (N, lm, c) in enumerate(trs)]
    x = torch.from_numpy(np.concatenate([v.reshape(-1) for v in xs])).cuda()
    return b, trs, xs, x


def check_forward(b, trs, xs, x):
    y = b.forward(x).cpu().numpy()
    offs = b.offsets()
    for k, (N, lm, c) in enumerate(trs):
        yk = y[offs[k]:offs[k] + sum(c) * N].reshape(-1, N)
        c0 = 0
        for l in range(lm + 1):
            if c[l]:
                xin = xs[k][c0:c0 + c[l]].astype(np.complex128)
                rows = sorted({0, 1, 2, 5, 31, 32, 33, 127, 128, N // 2, N - 1})
                ref = oracle.forward_rows(l, xin, rows)
                e = (np.abs(yk[c0:c0 + c[l]][:, rows] - ref).max(axis=1) / np.linalg.norm(xin, axis=1)).max()
                assert e < 1e-6, (N, l, e)
            c0 += c[l]


def test_batch_forward_matches_oracle_per_grid(lib):
    b, trs, xs, x = make(lib)
    info = b.info()
    assert info["bn_cap"] in (128, 192, 256) and all(v > 0 for v in info["tune_ms"].values())
    check_forward(b, trs, xs, x)
    b.close()


def test_every_tile_order_and_width(lib):
    """The pinned tile orders and widths give the oracle's forward and the same
    kinetic step (up to FP32 rounding order of the inverse's K walk)."""
    b, trs, xs, x = make(lib)
    b.set_tiles("transform-major", 256)
    ref = b.kinetic(x, 0.05)          # channels have unit norm: absolute error is relative
    for order in b.TILE_ORDERS:
        for cap in (128, 192, 256):
            b.set_tiles(order, cap)
            info = b.info()
            assert info["order"] == order and info["bn_cap"] == cap
            check_forward(b, trs, xs, x)
            e = (b.kinetic(x, 0.05) - ref).abs().max().item()
            assert e < 1e-6, (order, cap, e)
    b.close()


def test_batch_kinetic_matches_single_plan_and_graph(lib):
    b, trs, xs, x = make(lib)
    tau = 0.05
    y = b.kinetic(x, tau)
    offs = b.offsets()
    for k, (N, lm, c) in enumerate(trs):
        p = lib.Plan(N, N * DR, lm, fp64=False)
        ref = p.kinetic_grouped(c, torch.from_numpy(xs[k]).cuda(), tau)
        yk = y[offs[k]:offs[k] + sum(c) * N].reshape(-1, N)
        nrm = torch.linalg.vector_norm(torch.from_numpy(xs[k]).cuda(), dim=1)
        e = ((yk - ref).abs().amax(dim=1) / nrm).max().item()
        assert e < 1e-6, (N, e)
        p.close()
    out = torch.empty_like(x)
    g = b.capture_kinetic(x, tau, out)
    out.zero_()
    b.launch_graph(g)
    b.launch_graph(g)
    torch.cuda.synchronize()
    assert torch.equal(out, y)
    b.close()


def test_full_uneven_workload_sampled(lib):
    """64 transforms, N ~ U{512..8192 step 256}, l_max ~ U{8..64} (seed 0), 2l+1
    channels per l: forward outputs of the largest and a small transform on
    sampled rows against the oracle at their own N; kinetic norm conservation on
    every channel."""
    work = inputs.grouped_workload(0)
    trs = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in work]
    b = lib.Batch(trs, 0.1, autotune=False)
    xs = [inputs.gaussian_sum(300 + k, N, 0.1, c, dtype=torch.complex64, device="cuda").reshape(-1)
          for k, (N, lm, c) in enumerate(trs)]
    x = torch.cat(xs)
    y = b.forward(x)
    b.set_tiles("l-major/row-interleaved", 256)       # the same outputs from the interleaved tile list
    assert (b.forward(x) - y).abs().max().item() < 1e-6
    b.set_tiles("l-major", 256)
    offs = b.offsets()
    big = max(range(len(trs)), key=lambda i: trs[i][0] * 100 + trs[i][1])
    small = min(range(len(trs)), key=lambda i: trs[i][0])
    for k in (big, small):
        N, lm, c = trs[k]
        yk = y[offs[k]:offs[k] + sum(c) * N].reshape(-1, N).cpu().numpy()
        xk = x[offs[k]:offs[k] + sum(c) * N].reshape(-1, N).cpu().numpy().astype(np.complex128)
        c0 = 0
        for l in range(lm + 1):
            if l in (0, 1, lm // 2, lm):
                sel = [c0, c0 + c[l] - 1]
                rows = [0, 1, 31, 32, 200, N - 1]
                ref = oracle.forward_rows(l, xk[sel], rows)
                e = (np.abs(yk[sel][:, rows] - ref).max(axis=1) / np.linalg.norm(xk[sel], axis=1)).max()
                assert e < 1e-6, (N, l, e)
            c0 += c[l]
    z = b.kinetic(x, 0.05)
    torch.cuda.synchronize()
    start = 0
    worst = 0.0
    for k, (N, lm, c) in enumerate(trs):
        n = sum(c) * N
        a = x[start:start + n].reshape(-1, N).to(torch.complex128)
        bz = z[start:start + n].reshape(-1, N).to(torch.complex128)
        na, nb = torch.linalg.vector_norm(a, dim=1), torch.linalg.vector_norm(bz, dim=1)
        worst = max(worst, ((nb - na) / na).abs().max().item())
        start += n
    assert worst < 2e-6, worst
    b.close()


def test_interval_scheme_batch(lib):
    """DSBT_BATCH_INTERVAL: one interval-scheme plan per distinct grid (grids of
    2, 6, 4, 10 and 8 leaves), transforms on internal streams.  Forward against
    the oracle at each transform's own N, kinetic step against the dense batch,
    and a CUDA-graph replay (the fork-join over the internal streams) equal to
    the direct call."""
    trs = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in TRANSFORMS]
    trs[1][2][4] = 0
    xs = [inputs.gaussian_sum(20 + k, N, DR, c).astype(np.complex64) for k, (N, lm, c) in enumerate(trs)]
    x = torch.from_numpy(np.concatenate([v.reshape(-1) for v in xs])).cuda()
    b = lib.Batch(trs, DR, scheme="interval")
    assert b.info()["order"] is None
    check_forward(b, trs, xs, x)
    tau = 0.05
    y = b.kinetic(x, tau)
    dense = lib.Batch(trs, DR, autotune=False)
    yd = dense.kinetic(x, tau)
    dense.close()
    assert (y - yd).abs().max().item() < 2e-6          # unit-norm channels
    out = torch.empty_like(x)
    g = b.capture_kinetic(x, tau, out)
    out.zero_()
    b.launch_graph(g)
    b.launch_graph(g)
    torch.cuda.synchronize()
    assert torch.equal(out, y)
    with pytest.raises(lib.DSBTError):
        b.set_tiles("l-major", 256)
    b.close()


def test_interval_scheme_full_uneven_workload(lib):
    """The 64-transform workload on the interval scheme: sampled forward rows of
    the largest and a small transform against the oracle, kinetic norm drift on
    every channel."""
    work = inputs.grouped_workload(0)
    trs = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in work]
    b = lib.Batch(trs, 0.1, scheme="interval")
    xs = [inputs.gaussian_sum(300 + k, N, 0.1, c, dtype=torch.complex64, device="cuda").reshape(-1)
          for k, (N, lm, c) in enumerate(trs)]
    x = torch.cat(xs)
    del xs
    y = b.forward(x)
    offs = b.offsets()
    big = max(range(len(trs)), key=lambda i: trs[i][0] * 100 + trs[i][1])
    small = min(range(len(trs)), key=lambda i: trs[i][0])
    for k in (big, small):
        N, lm, c = trs[k]
        yk = y[offs[k]:offs[k] + sum(c) * N].reshape(-1, N).cpu().numpy()
        xk = x[offs[k]:offs[k] + sum(c) * N].reshape(-1, N).cpu().numpy().astype(np.complex128)
        c0 = 0
        for l in range(lm + 1):
            if l in (0, 1, lm // 2, lm):
                sel = [c0, c0 + c[l] - 1]
                rows = [0, 1, 31, 32, 200, N - 1]
                ref = oracle.forward_rows(l, xk[sel], rows)
                e = (np.abs(yk[sel][:, rows] - ref).max(axis=1) / np.linalg.norm(xk[sel], axis=1)).max()
                assert e < 1e-6, (N, l, e)
            c0 += c[l]
    del y
    z = b.kinetic(x, 0.05)
    torch.cuda.synchronize()
    start = 0
    worst = 0.0
    for k, (N, lm, c) in enumerate(trs):
        n = sum(c) * N
        a = x[start:start + n].reshape(-1, N).to(torch.complex128)
        bz = z[start:start + n].reshape(-1, N).to(torch.complex128)
        na, nb = torch.linalg.vector_norm(a, dim=1), torch.linalg.vector_norm(bz, dim=1)
        worst = max(worst, ((nb - na) / na).abs().max().item())
        start += n
    assert worst < 2e-6, worst
    b.close()
