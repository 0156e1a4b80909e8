"""The contractions the bench times, against the FP64 oracle at the sizes the
bench runs them (N = 4096, l <= 63, all m x batch 8 = 32768 complex64
channels, launched exactly as the bench launches them) and at the largest
grid (N = 8192, l_max = 64).

The oracle forms T_l row by row from the DLOP recurrence in binary128
(Sec. 2.4, Eqs. (38)-(43)), so any row is cheap but a whole N x N factor is
not.  Outputs are therefore checked where the oracle can compute them one by
one, and by properties that hold at any size:

* forward: b[rows] = T_l[rows] F_l psi on rows in every leaf and level of the
  interval tree (completion rows, both sides of each 128-row leaf boundary,
  the first and last rows), element by element;
* inverse: coefficient vectors that vanish outside a row set S with rows in
  every leaf give psi = F_l^T T_l[S]^T b[S] exactly, compared on all N samples;
* kinetic step: T_l F_l y = exp(-i k~^2 tau / 2) T_l F_l psi on the sampled
  rows (orthogonality, Eq. (25)), and the round trip on every channel.

Bar: max |gpu - oracle| / ||psi|| per channel <= 1e-6 (split precision),
1e-12 (FP64).
"""
import functools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1509_07115_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
TOL64 = 1e-12
TAU = 0.05


@functools.lru_cache(maxsize=2)
def _F(N, parity):
    return oracle.F_matrix(N, parity)


def T_rows(N, l, rows):
    """oracle.T_rows over threads (the C routine releases the GIL; each row is
    computed independently, so the result does not depend on the split)."""
    rows = np.asarray(rows)
    nt = max(1, min(16, os.cpu_count() or 1, rows.size // 8))
    if nt == 1:
        return oracle.T_rows(N, l, rows)
    parts = np.array_split(rows, nt)
    with ThreadPoolExecutor(nt) as ex:
        out = list(ex.map(lambda r: oracle.T_rows(N, l, r), parts))
    return np.concatenate(out)


def f_lines(l, x):
    """F_l x by the oracle's naive sums (F depends on the parity of l only)."""
    return oracle.apply(_F(x.shape[-1], l % 2), x)


def fwd_rows(l, x, rows):
    return f_lines(l, x) @ T_rows(x.shape[-1], l, rows).T


def sample_rows(N, l, seed):
    ne = oracle.n0(l) - oracle.p_of(l)          # completion rows n < n0_l (Sec. 2.5)
    fixed = {0, 1, ne - 1, ne, ne + 1, 31, 32, 63, 64, 127, 128, 255, 256, 1023, 1024, 2047, 2048,
             N - 129, N - 128, N - 2, N - 1}
    rng = np.random.default_rng(seed)
    fixed.update(int(v) for v in rng.integers(0, N, 4))
    return sorted(r for r in fixed if 0 <= r < N)


def leaf_rows(N, l, seed, per_leaf=3):
    """Row set S of the sparse inverse inputs: the completion rows, both rows
    at every leaf boundary and per_leaf random rows inside every 128-row leaf."""
    ne = oracle.n0(l) - oracle.p_of(l)
    rng = np.random.default_rng(seed)
    s = set(range(ne + 1))
    for j in range(N // 128):
        s.update((128 * j, 128 * j + 127))
        s.update(int(v) for v in 128 * j + rng.integers(0, 128, per_leaf))
    return np.array(sorted(s))


def worst(got, ref, norms):
    return float((np.abs(np.asarray(got) - np.asarray(ref)).max(axis=1) / np.asarray(norms)).max())


def group_slices(counts):
    c0 = 0
    for l, c in enumerate(counts):
        yield l, c0, c
        c0 += c


def sparse_batch(seed, counts, N, sets, dtype, device):
    """Batch of coefficient vectors, channel group l supported on sets[l]."""
    b = torch.zeros((sum(counts), N), dtype=dtype, device=device)
    for l, c0, c in group_slices(counts):
        if c:
            S = sets[l]
            v = inputs.sparse_coefficient_values(seed + l, c, S.size)
            b[c0:c0 + c][:, torch.as_tensor(S, device=device)] = torch.as_tensor(v, device=device).to(dtype)
    return b


def check_groups(counts, ls, x_np_of, got_of, ref_of, tol, what):
    for l, c0, c in group_slices(counts):
        if l not in ls or c == 0:
            continue
        sel = sorted({c0, c0 + c // 2, c0 + c - 1})
        x = x_np_of(sel)
        e = worst(got_of(sel), ref_of(l, x), np.linalg.norm(x, axis=1))
        assert e < tol, (what, l, e)


@pytest.fixture(scope="module")
def precision_plan(lib):
    """The bench's plan: N = 4096, r_max = 409.6, l <= 63, interval-scheme
    split contraction (DSBT_PLAN_FAST_SPLIT), no FP64 factors."""
    p = lib.Plan(4096, 409.6, 63, fp64=False, tf32x3=True, fast_split=True)
    yield p
    p.close()


LS_C3 = (0, 1, 2, 31, 32, 62, 63)


def test_precision_workload_forward_rows(precision_plan):
    N, counts = 4096, inputs.all_m_counts(63, 8)
    x = inputs.gaussian_sum(2, N, 0.1, counts, dtype=torch.complex64, device="cuda")
    b = precision_plan.forward_grouped(counts, x)
    torch.cuda.synchronize()
    assert precision_plan.device_status() == 0
    for l in LS_C3:
        rows = sample_rows(N, l, 100 + l)
        check_groups(counts, (l,), lambda s: x[s].cpu().numpy().astype(np.complex128),
                     lambda s: b[s].cpu().numpy()[:, rows], lambda l_, xs: fwd_rows(l_, xs, rows), TOL32,
                     "forward")


def test_precision_workload_inverse_sparse(precision_plan):
    N, counts = 4096, inputs.all_m_counts(63, 8)
    sets = [leaf_rows(N, l, 300 + l) for l in range(64)]
    b = sparse_batch(7, counts, N, sets, torch.complex64, "cuda")
    psi = precision_plan.inverse_grouped(counts, b)
    torch.cuda.synchronize()
    assert precision_plan.device_status() == 0
    for l in LS_C3:
        S = sets[l]
        TS = T_rows(N, l, S)

        def ref(l_, bs, S=S, TS=TS):
            return oracle.apply(_F(N, l_ % 2), bs[:, S] @ TS, transpose=True)
        check_groups(counts, (l,), lambda s: b[s].cpu().numpy().astype(np.complex128),
                     lambda s: psi[s].cpu().numpy(), ref, TOL32, "inverse")


def test_precision_workload_kinetic_and_round_trip(precision_plan):
    N, counts = 4096, inputs.all_m_counts(63, 8)
    x = inputs.gaussian_sum(3, N, 0.1, counts, dtype=torch.complex64, device="cuda")
    y = precision_plan.kinetic_grouped(counts, x, TAU)
    b = precision_plan.forward_grouped(counts, x)
    z = precision_plan.inverse_grouped(counts, b)
    torch.cuda.synchronize()
    assert precision_plan.device_status() == 0
    rt = (z - x).abs().amax(dim=1).max().item()           # unit-norm channels
    assert rt < 2 * TOL32, rt
    for l in LS_C3:
        rows = sample_rows(N, l, 200 + l)
        ph = np.exp(-0.5j * oracle.k_tilde(N, 409.6, l)[rows] ** 2 * TAU)
        for l_, c0, c in group_slices(counts):
            if l_ != l:
                continue
            sel = [c0, c0 + c // 2, c0 + c - 1]
            xs = x[sel].cpu().numpy().astype(np.complex128)
            ys = y[sel].cpu().numpy().astype(np.complex128)
            lhs = fwd_rows(l, ys, rows)
            rhs = fwd_rows(l, xs, rows) * ph
            assert worst(lhs, rhs, np.linalg.norm(xs, axis=1)) < TOL32, l


def test_largest_grid_l64_forward_inverse(lib):
    """N = 8192 (64 leaves, six tree levels), l_max = 64 (completion rows of
    degree 63 through the right intervals)."""
    N, lmax = 8192, 64
    counts = [1] * (lmax + 1)
    for l in (0, 1, 2, 31, 32, 63, 64):
        counts[l] = 3
    p = lib.Plan(N, 819.2, lmax, fp64=False, tf32x3=True, fast_split=True)
    x = inputs.gaussian_sum(4, N, 0.1, counts, dtype=torch.complex64, device="cuda")
    b = p.forward_grouped(counts, x)
    sets = [leaf_rows(N, l, 500 + l, per_leaf=2) for l in range(lmax + 1)]
    bs = sparse_batch(9, counts, N, sets, torch.complex64, "cuda")
    psi = p.inverse_grouped(counts, bs)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    for l in (0, 1, 2, 31, 32, 63, 64):
        rows = sample_rows(N, l, 600 + l)
        check_groups(counts, (l,), lambda s: x[s].cpu().numpy().astype(np.complex128),
                     lambda s: b[s].cpu().numpy()[:, rows], lambda l_, xs: fwd_rows(l_, xs, rows), TOL32,
                     "forward")
        S = sets[l]
        TS = T_rows(N, l, S)
        check_groups(counts, (l,), lambda s: bs[s].cpu().numpy().astype(np.complex128),
                     lambda s: psi[s].cpu().numpy(),
                     lambda l_, bb: oracle.apply(_F(N, l_ % 2), bb[:, S] @ TS, transpose=True), TOL32,
                     "inverse")
    p.close()


@pytest.mark.parametrize("N", [2048, 4096])
def test_fast64_high_l_against_oracle(lib, N):
    """DSBT_PLAN_FAST64 (FP64 interval scheme, degree-63 bases) on l = 31, 63:
    the kinetic step satisfies T_l F_l y = exp(-i k~^2 tau/2) T_l F_l psi on
    sampled rows to FP64 accuracy."""
    lmax = 63
    counts = [0] * (lmax + 1)
    for l in (0, 1, 31, 62, 63):
        counts[l] = 2
    p = lib.Plan(N, 0.1 * N, lmax, tf32x3=False, fast64=True)
    x = inputs.gaussian_sum(11, N, 0.1, counts)
    y = p.kinetic_grouped(counts, torch.from_numpy(x).cuda(), TAU).cpu().numpy()
    p.close()
    for l, c0, c in group_slices(counts):
        if c == 0:
            continue
        rows = sample_rows(N, l, 700 + l)
        ph = np.exp(-0.5j * oracle.k_tilde(N, 0.1 * N, l)[rows] ** 2 * TAU)
        lhs = fwd_rows(l, y[c0:c0 + c], rows)
        rhs = fwd_rows(l, x[c0:c0 + c], rows) * ph
        assert worst(lhs, rhs, np.linalg.norm(x[c0:c0 + c], axis=1)) < TOL64, (N, l)


@pytest.mark.parametrize("N", [4096, 8192])
def test_plan_rows_large_grids(lib, N):
    """Rows of the GPU-built FP64 T_l (difference equation in x) against the
    oracle's binary128 rows near n0_l, at leaf boundaries and in the last leaf."""
    p = lib.Plan(N, 0.1 * N, 64, tf32x3=False)
    for l in (32, 63, 64):
        ne = oracle.n0(l) - oracle.p_of(l)
        rows = [0, 1, ne - 1, ne, ne + 1, 127, 128, N // 2, N - 129, N - 128, N - 2, N - 1]
        T = p.get_T(l)[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        ref = T_rows(N, l, rows)
        assert np.abs(T - ref).max() < 1e-14, (N, l, np.abs(T - ref).max())
    p.close()


@pytest.mark.parametrize("cplx", [True, False])
def test_c2_fast64_forward_inverse_against_oracle(lib, cplx):
    """The FP64 configuration (N = 2048, r_max = 204.8, l <= 31, all m: 1024
    complex128 channels; or their real parts as FP64 lines) on a
    DSBT_PLAN_FAST64 plan, whose O(N l log N) contraction also serves the
    caller's interleaved and real layouts: sampled forward rows and sparse
    inverse inputs against the oracle at 1e-12, round trip on every channel."""
    N, lmax = 2048, 31
    counts = inputs.all_m_counts(lmax)
    x = inputs.gaussian_sum(1, N, 0.1, counts)
    if not cplx:
        x = x.real.copy()
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    p = lib.Plan(N, 204.8, lmax, tf32x3=False, fast64=True)
    b = p.forward_grouped(counts, torch.from_numpy(x).cuda())
    y = p.inverse_grouped(counts, b).cpu().numpy()
    bn = b.cpu().numpy()
    sets = [leaf_rows(N, l, 800 + l, per_leaf=2) for l in range(lmax + 1)]
    bs = sparse_batch(21, counts, N, sets, torch.complex128, "cuda")
    if not cplx:
        bs = bs.real.contiguous()
    psi = p.inverse_grouped(counts, bs).cpu().numpy()
    bs = bs.cpu().numpy()
    p.close()
    assert worst(y, x, np.linalg.norm(x, axis=1)) < TOL64
    for l, c0, c in group_slices(counts):
        if l not in (0, 1, 2, 15, 30, 31):
            continue
        sel = [c0, c0 + c - 1]
        rows = sample_rows(N, l, 900 + l)
        assert worst(bn[sel][:, rows], fwd_rows(l, x[sel], rows), np.linalg.norm(x[sel], axis=1)) < TOL64, l
        S = sets[l]
        ref = oracle.apply(_F(N, l % 2), bs[sel][:, S] @ T_rows(N, l, S), transpose=True)
        assert worst(psi[sel], ref, np.linalg.norm(bs[sel], axis=1)) < TOL64, l
