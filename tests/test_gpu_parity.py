"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Error metric (per channel): max |gpu - oracle| / ||psi||_2 (the transform is
orthogonal, so ||psi|| = ||b||).  Bars: FP64 path 1e-12, split-TF32 path 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1509_07115_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def rel_err(got, ref):
    got = np.asarray(got).reshape(-1, np.asarray(got).shape[-1])
    ref = np.asarray(ref).reshape(got.shape)
    nrm = np.linalg.norm(ref, axis=1)
    nrm[nrm == 0] = 1.0
    return float((np.abs(got - ref).max(axis=1) / nrm).max())


def rel_err_sampled(got, ref, norms):
    """max |got - ref| / ||psi|| for sampled outputs of channels with norms."""
    got = np.asarray(got)
    ref = np.asarray(ref).reshape(got.shape)
    return float((np.abs(got - ref).max(axis=1) / np.asarray(norms)).max())


def oracle_grouped(fn, counts, x):
    out = np.empty_like(x)
    c0 = 0
    for l, c in enumerate(counts):
        if c:
            out[c0:c0 + c] = fn(l, x[c0:c0 + c])
        c0 += c
    return out


@pytest.fixture(scope="module")
def plan256(lib):
    p = lib.Plan(256, 25.6, 64)
    yield p
    p.close()


def test_plan_factors_match_oracle(plan256):
    info = plan256.info()
    assert info["check_err"] < 1e-13
    for l in (0, 1, 2, 3, 8, 17, 31, 32, 63, 64):
        T = plan256.get_T(l).cpu().numpy()
        ref = oracle.T_matrix(256, l)
        assert np.abs(T - ref).max() < 1e-14, l


def test_plan_factor_rows_large_N(lib):
    p = lib.Plan(2048, 204.8, 31, tf32x3=False)
    for l in (1, 16, 31):
        T = p.get_T(l).cpu().numpy()
        rows = [0, 1, 15, 16, 17, 100, 1023, 2047]
        ref = oracle.T_rows(2048, l, rows)
        assert np.abs(T[rows] - ref).max() < 1e-14, l
    p.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.float64])
def test_fp64_grouped_forward_inverse(plan256, dtype):
    counts = [(2 * l + 1) for l in range(9)] + [0] * 56
    counts[3] = 0          # an empty group in the middle
    counts[8] = 70         # several 64-line tiles with a ragged tail
    total = sum(counts)
    x = inputs.gaussian_sum(5, 256, 0.1, counts)
    if dtype == torch.float64:
        x = x.real.copy()
    xt = torch.from_numpy(x).cuda()
    b = plan256.forward_grouped(counts, xt)
    ref = oracle_grouped(oracle.forward, counts, x)
    assert rel_err(b.cpu().numpy(), ref) < TOL64
    y = plan256.inverse_grouped(counts, b)
    refi = oracle_grouped(oracle.inverse, counts, ref)
    assert rel_err(y.cpu().numpy(), refi) < TOL64
    assert rel_err(y.cpu().numpy(), x) < TOL64
    assert total == xt.shape[0]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.float32])
def test_tf32x3_grouped_forward_inverse(plan256, dtype):
    counts = [(2 * l + 1) * 3 for l in range(65)]
    counts[5] = 0
    counts[64] = 200       # > 256 real lines: two column tiles, ragged
    x = inputs.gaussian_sum(6, 256, 0.1, counts)
    if dtype == torch.float32:
        x = x.real.copy()
    x = x.astype(np.complex64 if dtype == torch.complex64 else np.float32)
    xt = torch.from_numpy(x).cuda()
    b = plan256.forward_grouped(counts, xt)
    x64 = x.astype(np.complex128 if dtype == torch.complex64 else np.float64)
    ref = oracle_grouped(oracle.forward, counts, x64)
    e = rel_err(b.cpu().numpy(), ref)
    assert e < TOL32, e
    y = plan256.inverse_grouped(counts, torch.from_numpy(ref.astype(x.dtype)).cuda())
    refi = oracle_grouped(oracle.inverse, counts, ref)
    e = rel_err(y.cpu().numpy(), refi)
    assert e < TOL32, e
    assert plan256.device_status() == 0


def test_single_l_calls_and_empty(plan256):
    rng = np.random.default_rng(7)
    for l, n in [(0, 1), (1, 3), (4, 1), (63, 2), (64, 5)]:
        x = (rng.standard_normal((n, 256)) + 1j * rng.standard_normal((n, 256)))
        ref = oracle.forward(l, x)
        b = plan256.forward(l, torch.from_numpy(x).cuda())
        assert rel_err(b.cpu().numpy(), ref) < TOL64
        b32 = plan256.forward(l, torch.from_numpy(x.astype(np.complex64)).cuda())
        assert rel_err(b32.cpu().numpy(), ref) < TOL32
        xi = plan256.inverse(l, torch.from_numpy(ref).cuda())
        assert rel_err(xi.cpu().numpy(), x) < TOL64
    # zero channels: a no-op that succeeds
    e = torch.empty((0, 256), dtype=torch.complex128, device="cuda")
    assert plan256.forward(3, e).shape == (0, 256)


def test_kinetic_step_matches_oracle(plan256):
    counts = [1] * 65
    counts[10] = 4
    x = inputs.gaussian_sum(8, 256, 0.1, counts)
    tau = 0.05
    dk = np.pi / 25.6
    ref = np.empty_like(x)
    c0 = 0
    for l, c in enumerate(counts):
        kt = oracle.k_tilde(256, 25.6, l)
        b = oracle.forward(l, x[c0:c0 + c]) * np.exp(-0.5j * kt * kt * tau)
        ref[c0:c0 + c] = oracle.inverse(l, b)
        c0 += c
    y = plan256.kinetic_grouped(counts, torch.from_numpy(x).cuda(), tau)
    assert rel_err(y.cpu().numpy(), ref) < TOL64
    y32 = plan256.kinetic_grouped(counts, torch.from_numpy(x.astype(np.complex64)).cuda(), tau)
    assert rel_err(y32.cpu().numpy(), ref) < 3 * TOL32


def test_orbital_config_real_fp64(lib):
    """N = 256, r_max = 20, l = 0..4, one real Gaussian orbital per l."""
    p = lib.Plan(256, 20.0, 4, tf32x3=False)
    xs, _ = inputs.orbital(0, 256, 20.0, range(5))
    x = np.concatenate(xs)
    b = p.forward_grouped([1] * 5, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = np.concatenate([oracle.forward(l, xs[l]) for l in range(5)])
    assert rel_err(b, ref) < TOL64
    y = p.inverse_grouped([1] * 5, torch.from_numpy(b).cuda()).cpu().numpy()
    assert rel_err(y, x) < TOL64
    p.close()


def test_full_size_fp64_config_sampled(lib):
    """N = 2048, r_max = 204.8, l <= 31, all m (1024 complex128 channels):
    sampled outputs against the oracle, round trip and norm on all channels."""
    N, lmax = 2048, 31
    counts = inputs.all_m_counts(lmax)
    p = lib.Plan(N, 204.8, lmax, tf32x3=False)
    x = inputs.gaussian_sum(1, N, 0.1, counts)
    xt = torch.from_numpy(x).cuda()
    b = p.forward_grouped(counts, xt)
    bn = b.cpu().numpy()
    rows = [0, 1, 7, 15, 16, 300, 1024, 2047]
    c0 = 0
    for l, c in enumerate(counts):
        if l in (0, 1, 2, 15, 30, 31):
            sel = [c0, c0 + c - 1]
            ref = oracle.forward_rows(l, x[sel], rows)
            assert rel_err_sampled(bn[sel][:, rows], ref, np.linalg.norm(x[sel], axis=1)) < TOL64, l
        c0 += c
    assert np.allclose(np.linalg.norm(bn, axis=1), 1.0, atol=1e-12)
    y = p.inverse_grouped(counts, b).cpu().numpy()
    assert rel_err(y, x) < TOL64
    p.close()


def test_full_size_precision_config_sampled(lib):
    """N = 4096, l <= 63, all m x batch 8 (32768 complex64 channels): sampled
    outputs against the oracle, round-trip error and norm drift on every channel."""
    N, lmax, batch = 4096, 63, 8
    counts = inputs.all_m_counts(lmax, batch)
    p = lib.Plan(N, 409.6, lmax, fp64=False)
    xt = inputs.gaussian_sum(2, N, 0.1, counts, dtype=torch.complex64, device="cuda")
    b = p.forward_grouped(counts, xt)
    y = p.inverse_grouped(counts, b)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    rt = ((y - xt).abs().amax(dim=1)).max().item()
    assert rt < 2 * TOL32, rt
    # norm drift |(||b|| - ||psi||)| / ||psi|| of the split-TF32 forward (reported
    # quantity; the truncating tensor-core accumulation biases it slightly low)
    nx = torch.linalg.vector_norm(xt.to(torch.complex128), dim=1)
    drift = ((torch.linalg.vector_norm(b.to(torch.complex128), dim=1) - nx) / nx).abs().max().item()
    assert drift < 2 * TOL32, drift
    rows = [0, 1, 31, 32, 33, 1000, 4095]
    c0 = 0
    for l, c in enumerate(counts):
        if l in (0, 1, 2, 31, 62, 63):
            sel = [c0, c0 + c // 2, c0 + c - 1]
            xs = xt[sel].cpu().numpy().astype(np.complex128)
            ref = oracle.forward_rows(l, xs, rows)
            e = rel_err_sampled(b[sel].cpu().numpy()[:, rows], ref, np.linalg.norm(xs, axis=1))
            assert e < TOL32, (l, e)
        c0 += c
    p.close()


@pytest.mark.parametrize("N", [768, 1280, 1536, 2304, 2816, 3840, 5376, 6400, 6912, 7936])
def test_non_power_of_two_grids(lib, N):
    """N = 256 q, q not a power of two (radix-16 stages, a radix-2 stage for
    q = 6, and one radix-Q stage for the odd part Q of q: primes 3, 5, 11, 31
    and composites 9, 15, 21, 25, 27): both precision paths against the oracle
    on sampled rows, and the round trip on all channels."""
    lmax = 9
    counts = [1] * (lmax + 1)
    counts[3] = 2
    p = lib.Plan(N, 0.1 * N, lmax)
    x = inputs.gaussian_sum(9, N, 0.1, counts)
    nrm = np.linalg.norm(x, axis=1)
    b64 = p.forward_grouped(counts, torch.from_numpy(x).cuda()).cpu().numpy()
    b32 = p.forward_grouped(counts, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    rows = [0, 1, 5, 6, 300, N // 2 + 7, N - 1]
    c0 = 0
    for l, c in enumerate(counts):
        ref = oracle.forward_rows(l, x[c0:c0 + c], rows)
        assert rel_err_sampled(b64[c0:c0 + c][:, rows], ref, nrm[c0:c0 + c]) < TOL64, (N, l)
        assert rel_err_sampled(b32[c0:c0 + c][:, rows], ref, nrm[c0:c0 + c]) < TOL32, (N, l)
        c0 += c
    y64 = p.inverse_grouped(counts, torch.from_numpy(b64).cuda()).cpu().numpy()
    assert rel_err(y64, x) < TOL64
    y32 = p.inverse_grouped(counts, torch.from_numpy(b32).cuda()).cpu().numpy()
    assert rel_err(y32, x) < 2 * TOL32
    p.close()
