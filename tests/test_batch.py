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


def test_batch_forward_matches_oracle_per_grid(lib):
    b, trs, xs, x = make(lib)
    info = b.info()
    assert info["bn_cap"] in (128, 192, 256) and all(v > 0 for v in info["tune_ms"].values())
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
