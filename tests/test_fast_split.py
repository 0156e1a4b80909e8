"""Split-precision tensor-core contractions through the interval scheme
(DSBT_PLAN_FAST_SPLIT, csrc/fast_split.cu): the near band of T_l per 128-row
leaf plus the far field through 64 basis functions per used dyadic interval,
operands as scaled FP16 pairs.  Same results as the FP64 contraction with the
dense T_l within the split-precision bar (1e-6 of the channel norm), for every
l (odd l carries the m = 0 weight) and grids of 2 to 64 leaves."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1509_07115_gb300 import dsbt, inputs


def test_fast_split_flag_rules():
    lib = dsbt.load()
    h = ctypes.c_void_p()
    assert lib.dsbt_plan_create(300, 30.0, 4, dsbt.DSBT_PLAN_FAST_SPLIT | dsbt.DSBT_PLAN_TF32X3, None,
                                ctypes.byref(h)) == -1          # N not a multiple of 256
    assert lib.dsbt_plan_create(8448, 844.8, 4, dsbt.DSBT_PLAN_FAST_SPLIT, None,
                                ctypes.byref(h)) == -1          # 66 leaves, past the largest grid


@pytest.mark.gpu
def test_fast_plan_without_dense_split_factors(lib):
    """DSBT_PLAN_FAST_TF32 alone (no dense split copies of T_l, no FP64
    factors kept) serves FP32 calls; FP64 calls are refused."""
    N, lmax = 1024, 12
    counts = [2] * (lmax + 1)
    x = inputs.gaussian_sum(3, N, 0.1, counts)
    nrm = np.linalg.norm(x, axis=1)
    full = lib.Plan(N, 0.1 * N, lmax, fp64=True, tf32x3=False)
    ref = full.forward_grouped(counts, torch.from_numpy(x).cuda()).cpu().numpy()
    full.close()
    p = lib.Plan(N, 0.1 * N, lmax, fp64=False, tf32x3=False, fast_split=True)
    b = p.forward_grouped(counts, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(b, ref, nrm) < 1e-6
    with pytest.raises(lib.DSBTError):
        p.forward_grouped(counts, torch.from_numpy(x).cuda())
    p.close()


def rel(a, b, nrm):
    return (np.abs(a - b).max(axis=1) / nrm).max()


def counts_for(lmax):
    c = [1] * (lmax + 1)
    for l in (0, 1, 2, 3, 31, 32, 33, lmax - 1, lmax):
        c[l] = 3
    return c


@pytest.mark.gpu
@pytest.mark.parametrize("N", [256, 1024, 4096])
def test_fast_split_matches_fp64(lib, N):
    r_max, lmax, tau = N * 0.1, 63, 0.05
    counts = counts_for(lmax)
    x = inputs.gaussian_sum(70 + N, N, r_max / N, counts)
    nrm = np.linalg.norm(x, axis=1)
    plan = lib.Plan(N, r_max, lmax, fp64=True, tf32x3=True, fast_split=True)
    x128 = torch.from_numpy(x).cuda()
    x64 = x128.to(torch.complex64)
    ref_b = plan.forward_grouped(counts, x128).cpu().numpy()
    b = plan.forward_grouped(counts, x64).cpu().numpy()
    assert rel(b, ref_b, nrm) < 1e-6
    ref_f = plan.inverse_grouped(counts, torch.from_numpy(ref_b).cuda()).cpu().numpy()
    f = plan.inverse_grouped(counts, torch.from_numpy(ref_b).cuda().to(torch.complex64)).cpu().numpy()
    assert rel(f, ref_f, nrm) < 1e-6
    assert rel(ref_f, x, nrm) < 1e-12                            # the FP64 reference round trip
    ref_k = plan.kinetic_grouped(counts, x128, tau).cpu().numpy()
    k = plan.kinetic_grouped(counts, x64, tau).cpu().numpy()
    assert rel(k, ref_k, nrm) < 1e-6
    plan.close()


@pytest.mark.gpu
def test_fast_split_error_close_to_dense_tf32(lib):
    """The interval scheme adds no error of its own beyond the split-TF32
    rounding: its deviation from FP64 stays within 2x of the dense split-TF32
    contraction's on the same input."""
    N, r_max, lmax = 2048, 204.8, 63
    counts = counts_for(lmax)
    x = inputs.gaussian_sum(91, N, r_max / N, counts)
    nrm = np.linalg.norm(x, axis=1)
    x128 = torch.from_numpy(x).cuda()
    fast = lib.Plan(N, r_max, lmax, fp64=True, tf32x3=True, fast_split=True)
    dense = lib.Plan(N, r_max, lmax, fp64=False, tf32x3=True)
    ref = fast.forward_grouped(counts, x128).cpu().numpy()
    e_fast = rel(fast.forward_grouped(counts, x128.to(torch.complex64)).cpu().numpy(), ref, nrm)
    e_dense = rel(dense.forward_grouped(counts, x128.to(torch.complex64)).cpu().numpy(), ref, nrm)
    fast.close()
    dense.close()
    assert e_fast < max(2.0 * e_dense, 2e-7), (e_fast, e_dense)


@pytest.mark.gpu
def test_fast_split_real_lines_and_edges(lib):
    """Real (DSBT_F32) channels, l_max = 64 (the largest: right slots of the
    completion rows at degree 63) and the largest grid N = 8192 (64 leaves,
    six levels) against the FP64 path of the same plan."""
    for N, lmax, counts in ((8192, 8, [2, 1, 1, 1, 1, 1, 1, 1, 2]),
                            (512, 64, [1] * 60 + [2, 1, 1, 2, 3])):
        r_max = N * 0.1
        plan = lib.Plan(N, r_max, lmax, fp64=True, tf32x3=True, fast_split=True)
        x = inputs.gaussian_sum(5 + N, N, r_max / N, counts).real.copy()
        nrm = np.linalg.norm(x, axis=1)
        ref = plan.forward_grouped(counts, torch.from_numpy(x).cuda()).cpu().numpy()
        b = plan.forward_grouped(counts, torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
        assert rel(b, ref, nrm) < 1e-6, (N, lmax)
        f = plan.inverse_grouped(counts, torch.from_numpy(ref.astype(np.float32)).cuda()).cpu().numpy()
        assert rel(f, x, nrm) < 1e-6, (N, lmax)
        plan.close()


@pytest.mark.gpu
def test_fast_split_host_streamed_matches_device(lib):
    """The host-streamed kinetic step (chunks that cut l groups) runs the
    interval scheme on every chunk: identical to the device call."""
    N, r_max, lmax = 1024, 102.4, 20
    counts = [3] * (lmax + 1)
    x = inputs.gaussian_sum(17, N, r_max / N, counts).astype(np.complex64)
    plan = lib.Plan(N, r_max, lmax, fp64=False, tf32x3=True, fast_split=True)
    dev = plan.kinetic_grouped(counts, torch.from_numpy(x).cuda(), 0.05).cpu().numpy()
    xh = torch.from_numpy(x).pin_memory()
    out = plan.kinetic_grouped_host(counts, xh, 0.05, chunks=5)
    torch.cuda.synchronize()
    plan.close()
    assert np.array_equal(out.numpy(), dev)


@pytest.mark.gpu
def test_fast_split_kinetic_with_corrected_momenta(lib):
    """DSBT_PLAN_KCORR with the interval scheme: the kinetic phase per (l, n)
    (the corrected momenta of Sec. 3) in the forward-rows epilogue, against the
    FP64 path of the same plan."""
    N, r_max, lmax, tau = 1024, 102.4, 40, 0.05
    counts = [2] * (lmax + 1)
    x = inputs.gaussian_sum(23, N, r_max / N, counts)
    nrm = np.linalg.norm(x, axis=1)
    plan = lib.Plan(N, r_max, lmax, fp64=True, tf32x3=True, kcorr=True, fast_split=True)
    ref = plan.kinetic_grouped(counts, torch.from_numpy(x).cuda(), tau).cpu().numpy()
    k = plan.kinetic_grouped(counts, torch.from_numpy(x.astype(np.complex64)).cuda(), tau).cpu().numpy()
    plan.close()
    assert rel(k, ref, nrm) < 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("N", [768, 1280, 2304, 6400, 7936])
def test_fast_split_any_leaf_count(lib, N):
    """Grids whose leaf count N / 128 is not a power of two (6, 10, 18, 50, 62
    leaves): the used intervals, the right intervals of the completion rows and
    the partial siblings at the right edge, against the FP64 path of the same
    plan (forward, inverse, kinetic step) and the oracle on sampled rows."""
    import oracle
    lmax = 40 if N <= 2304 else 64
    counts = [1] * (lmax + 1)
    for l in (0, 1, 2, 3, 17, lmax - 1, lmax):
        counts[l] = 3
    x = inputs.gaussian_sum(90 + N // 256, N, 0.1, counts)
    nrm = np.linalg.norm(x, axis=1)
    plan = lib.Plan(N, 0.1 * N, lmax, fp64=True, tf32x3=False, fast_split=True)
    x128 = torch.from_numpy(x).cuda()
    x64 = x128.to(torch.complex64)
    ref_b = plan.forward_grouped(counts, x128).cpu().numpy()
    b = plan.forward_grouped(counts, x64).cpu().numpy()
    assert rel(b, ref_b, nrm) < 1e-6
    f = plan.inverse_grouped(counts, torch.from_numpy(ref_b).cuda().to(torch.complex64)).cpu().numpy()
    assert rel(f, x, nrm) < 1e-6
    ref_k = plan.kinetic_grouped(counts, x128, 0.05).cpu().numpy()
    k = plan.kinetic_grouped(counts, x64, 0.05).cpu().numpy()
    assert rel(k, ref_k, nrm) < 1e-6
    plan.close()
    rows = sorted({0, 1, 30, 127, 128, 129, N // 2, N - 129, N - 128, N - 1})
    c0 = 0
    for l, c in enumerate(counts):
        if l in (0, 1, lmax):
            ref = oracle.forward_rows(l, x[c0:c0 + c], rows)
            assert rel(b[c0:c0 + c][:, rows], ref, nrm[c0:c0 + c]) < 1e-6, (N, l)
        c0 += c


@pytest.mark.gpu
@pytest.mark.parametrize("N", [2048, 6400])
def test_fast_split_tile_order_does_not_change_results(lib, N):
    """Each direction is one launch in which a unit's row tiles wait on a
    device counter for its moment (weight) tiles; the lag between the two in
    the tile order only moves work in time.  Lags 1, 2, 5 and the plain order
    (every first tile, then every row tile) give bit-identical forward, inverse
    and kinetic results, within the split-precision bar of the FP64 path; the
    status word shows no wait that gave up.  Groups span up to five column
    tiles of 256 lines, with l = 0 (no moments) and empty groups among them;
    N = 6400 has 50 leaves (partial siblings, greedy right intervals).  Real
    lines go through the same launches."""
    r_max, lmax = 0.1 * N, 24
    counts = [0 if l in (5, 6) else (160 if l % 3 == 0 else 7) for l in range(lmax + 1)]
    x = inputs.gaussian_sum(57, N, r_max / N, counts)
    nrm = np.linalg.norm(x, axis=1)
    plan = lib.Plan(N, r_max, lmax, fp64=True, tf32x3=False, fast_split=True)
    x128 = torch.from_numpy(x).cuda()
    x64 = x128.to(torch.complex64)
    ref_b = plan.forward_grouped(counts, x128).cpu().numpy()
    ref_k = plan.kinetic_grouped(counts, x128, 0.05).cpu().numpy()
    out = {}
    for lag in (1, 2, 5, 1 << 20):
        plan.set_fast_lag(lag)
        b = plan.forward_grouped(counts, x64)
        f = plan.inverse_grouped(counts, b)
        k = plan.kinetic_grouped(counts, x64, 0.05)
        torch.cuda.synchronize()
        assert plan.device_status() == 0, lag
        out[lag] = [t.cpu().numpy() for t in (b, f, k)]
    plan.set_fast_lag(4)
    with pytest.raises(lib.DSBTError):
        plan.set_fast_lag(0)
    plan.close()
    b, f, k = out[1]
    assert rel(b, ref_b, nrm) < 1e-6
    assert rel(f, x, nrm) < 1e-6
    assert rel(k, ref_k, nrm) < 1e-6
    for lag in (2, 5, 1 << 20):
        for a, c in zip(out[1], out[lag]):
            assert np.array_equal(a, c), lag
    # real lines (DSBT_F32), lag 1 against the plain order
    xr = torch.from_numpy(x.real.astype(np.float32)).cuda()
    plan = lib.Plan(N, r_max, lmax, fp64=False, tf32x3=False, fast_split=True)
    res = []
    for lag in (1, 1 << 20):
        plan.set_fast_lag(lag)
        br = plan.forward_grouped(counts, xr)
        res.append((br.cpu().numpy(), plan.inverse_grouped(counts, br).cpu().numpy()))
    assert plan.device_status() == 0
    plan.close()
    for a, c in zip(res[0], res[1]):
        assert np.array_equal(a, c)
