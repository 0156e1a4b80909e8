"""Pins the FP64 oracle (oracle/) to facts the paper and mathematics fix, with no
GPU.  Each test names the passage it checks.  A plausible mistake in the oracle
(a dropped term, a sign, an index shift, a transposed operand) breaks at least
one of these.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft as sfft
from scipy import integrate
from scipy.special import eval_legendre, legendre, spherical_jn

import oracle
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def s_l(l):
    """Sign (-1)^{ceil(l/2)} relating plain sin/cos F to the paper's c~ (Eq. (6))."""
    return -1.0 if ((l + 1) // 2) % 2 else 1.0


# ------------------------------------------------------------ DLOP (Sec. 2.3)

def test_dlop_matches_exact_golden():
    """Binary128 recurrence vs the exact falling-factorial sum (Eq. (29)),
    stored in tests/golden/dlop_exact.txt."""
    worst = 0.0
    with open(os.path.join(GOLDEN, "dlop_exact.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            l, M, x, num, den = (int(t) for t in line.split())
            ref = num / den
            got = oracle.dlop(l, M, x)
            worst = max(worst, abs(got - ref) / max(1.0, abs(ref)))
    assert worst < 1e-15


def test_dlop_orthogonality_and_norm():
    """Eq. (27): sum_{i=0}^M P_l P_k = N(l, M) delta_lk, Eq. (28) for N(l, M)."""
    M = 40
    L = 12
    P = np.array([[oracle.dlop(l, M, i) for i in range(M + 1)] for l in range(L + 1)])
    G = P @ P.T
    nrm = np.array([oracle.dlop_norm(l, M) for l in range(L + 1)])
    assert np.allclose(np.diag(G), nrm, rtol=1e-13, atol=0)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12 * nrm.max()
    # the exact-rational norm formula agrees with an exact sum
    for l in range(0, 7):
        s = sum(exact.dlop(l, 11, i) ** 2 for i in range(12))
        assert s == exact.dlop_norm(l, 11)


def test_dlop_parity():
    """Eq. (A.3): P_l(i, M) = (-1)^l P_l(M - i, M)."""
    for l in range(0, 9):
        for M in (9, 20):
            for i in range(M + 1):
                a, b = oracle.dlop(l, M, i), oracle.dlop(l, M, M - i)
                assert abs(a - (-1) ** l * b) < 1e-13


def test_dlop_vs_legendre_first_order():
    """Eq. (30) states P_l(i, N) -> P_l(1 - 2i/N) at O(N^-2).  The explicit sum
    gives O(N^-1): for l = 2 the difference is exactly
    l(2,2) [i(i-1)/(N(N-1)) - (i/N)^2] = -6 i (N-i) / (N^2 (N-1)).
    Pinned here as the exact first-order term, and the rate as ~2 per doubling."""
    for N in (16, 40):
        for i in range(N + 1):
            d = oracle.dlop(2, N, i) - eval_legendre(2, 1 - 2 * i / N)
            assert abs(d - (-6.0 * i * (N - i) / (N * N * (N - 1)))) < 1e-14
    errs = []
    for N in (64, 128, 256):
        i = np.arange(N + 1)
        P = np.array([oracle.dlop(5, N, int(x)) for x in i])
        errs.append(np.abs(P - eval_legendre(5, 1 - 2 * i / N)).max())
    assert 1.9 < errs[0] / errs[1] < 2.2 and 1.9 < errs[1] / errs[2] < 2.2


def test_ddlop_to_derivative_third_order():
    """Eq. (36): P'_l(i, N) = d/di P_l(1 - 2i/N) + O(N^-3)  (ratio ~8)."""
    for l in (2, 3, 5):
        errs = []
        dP = np.polyder(legendre(l))
        for N in (64, 128, 256):
            i = np.arange(N + 1)
            d = np.array([oracle.ddlop(l, N, int(x)) for x in i])
            errs.append(np.abs(d + 2.0 / N * dP(1 - 2 * i / N)).max())
        assert 7.5 < errs[0] / errs[1] < 8.5 and 7.5 < errs[1] / errs[2] < 8.5


def test_sum_ddlop_poly_identity_exact():
    """Eq. (32): sum_{i=0}^M P'_l(i, M) p(i) w_i(M) = (-1)^l p(M) - p(0) for
    polynomials of order below l (proved in the appendix, Eqs. (A.1)-(A.7)).
    Exact rationals, and the oracle's DDLOP to 1e-12."""
    for l in range(1, 7):
        for M in (l + 1, l + 4, 12):
            wts = [Fraction(1, 2) if i in (0, M) else Fraction(1) for i in range(M + 1)]
            for s in range(0, l):
                lhs = sum(exact.ddlop(l, M, i) * Fraction(i) ** s * wts[i] for i in range(M + 1))
                rhs = (-1) ** l * Fraction(M) ** s - (1 if s == 0 else 0)
                assert lhs == rhs
                lhs_f = sum(oracle.ddlop(l, M, i) * float(i) ** s * float(wts[i]) for i in range(M + 1))
                assert abs(lhs_f - float(rhs)) < 1e-12 * max(1.0, float(M) ** s)


# ------------------------------------------------------------ T_l (Sec. 2.4, 2.5)

def test_exact_gram_is_diagonal():
    """Eq. (41): rows of I - L are mutually orthogonal (exact), and orthogonal to
    the extra rows of Eq. (43); extra-row squared norms are N(2n-p, 2N_l)/2,
    which is the closed-form alpha_n stated after Eq. (44)."""
    for N in (5, 8):
        for l in range(0, 7):
            if exact.n0(l) > N:
                continue
            G = exact.gram(N, l)
            p = exact.p_of(l)
            for a in range(N):
                for b in range(N):
                    if a != b:
                        assert G[a][b] == 0, (N, l, a, b)
            Nl = N + p - 1
            for n in range(p, exact.n0(l)):
                assert G[n - p][n - p] == exact.dlop_norm(2 * n - p, 2 * Nl) / 2


def test_T_matches_exact_rows_golden():
    """Oracle T_l against the exact rational rows of tests/golden/t_rows_exact.txt
    (element by element, including signs and the theta(0)=1/2 diagonal)."""
    cache = {}
    with open(os.path.join(GOLDEN, "t_rows_exact.txt")) as fh:
        lines = [ln for ln in fh if not ln.startswith("#")]
    k = 0
    checked = 0
    while k < len(lines):
        _, N, l, r, gn, gd = lines[k].split()
        N, l, r = int(N), int(l), int(r)
        g = int(gn) / int(gd)
        ents = [Fraction(t) for t in lines[k + 1].split()]
        p = exact.p_of(l)
        if (N, l) not in cache:
            cache[(N, l)] = oracle.T_matrix(N, l)
        T = cache[(N, l)]
        for c in range(N):
            wm = 0.5 if c + p == 0 else 1.0
            ref = float(ents[c]) * np.sqrt(wm) / np.sqrt(g)
            assert abs(T[r, c] - ref) < 2e-15, (N, l, r, c, T[r, c], ref)
        checked += 1
        k += 2
    assert checked > 50


@pytest.mark.parametrize("N,ls", [(64, range(0, 20)), (256, (0, 1, 2, 7, 16, 31, 32, 63, 64))])
def test_T_orthogonal(N, ls):
    """T T^T = I (Sec. 2.4-2.5) to FP64 accuracy, including l close to 2 n0."""
    for l in ls:
        T = oracle.T_matrix(N, l)
        err = np.abs(T @ T.T - np.eye(N)).max()
        assert err < 1e-13, (N, l, err)


def test_T_l0_identity_l1_closed_form():
    """l = 0: T = I (c_0 = c~_0 below Eq. (7)).  l = 1 (derived from Eqs. (34),
    (38)-(39) with P_1(i, M) = 1 - 2i/M): L_nm = theta(n-m) sqrt(w_m)/n,
    alpha_n = 2n / sqrt(4n^2 - 1); extra row n = 0: alpha_0 sqrt(w_m),
    alpha_0 = sqrt(2 / (2N - 1))."""
    N = 33
    assert np.array_equal(oracle.T_matrix(N, 0), np.eye(N))
    T = oracle.T_matrix(N, 1)
    ref = np.zeros((N, N))
    wm = np.ones(N)
    wm[0] = 0.5
    ref[0, :] = np.sqrt(2.0 / (2 * N - 1)) * np.sqrt(wm)
    for n in range(1, N):
        a = 2 * n / np.sqrt(4.0 * n * n - 1)
        for m in range(N):
            th = 1.0 if m < n else (0.5 if m == n else 0.0)
            L = th * np.sqrt(wm[m]) / n
            ref[n, m] = a * ((1.0 if m == n else 0.0) - L)
    assert np.abs(T - ref).max() < 1e-15


# ------------------------------------------------------------ F_l (Sec. 2.2)

def test_F_matches_library_dst_dct():
    """Eq. (16): even l -> orthonormal DST-II, odd l -> orthonormal DCT-II."""
    rng = np.random.default_rng(1)
    for N in (8, 37, 64):
        x = rng.standard_normal((3, N))
        for l in (0, 1, 2, 5):
            y = oracle.apply(oracle.F_matrix(N, l), x)
            ref = (sfft.dst if l % 2 == 0 else sfft.dct)(x, type=2, norm="ortho", axis=-1)
            assert np.abs(y - ref).max() < 1e-14


def test_l0_forward_is_dst():
    """l = 0 DSBT = orthonormal sine transform (T_0 = I)."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 48)) + 1j * rng.standard_normal((4, 48))
    b = oracle.forward(0, x)
    ref = sfft.dst(x.real, type=2, norm="ortho") + 1j * sfft.dst(x.imag, type=2, norm="ortho")
    assert np.abs(b - ref).max() < 1e-14


# ------------------------------------------------------------ DSBT vs physics (Sec. 3)

def gaussian_case(l, rmax, dr, alpha):
    N = int(round(rmax / dr))
    r = (np.arange(1, N + 1) - 0.5) * dr
    psi = r ** (l + 1) * np.exp(-alpha * r * r) * np.sqrt(dr)
    p = oracle.p_of(l)
    n = np.arange(N) + p
    dk = np.pi / rmax
    k = n * dk
    wn = np.where(n == 0, 0.5, 1.0) * dk
    c = k ** (l + 1) * np.exp(-k * k / (4 * alpha)) / (2 * alpha) ** (l + 1.5)
    return psi, n, k, wn, c


def test_gaussian_closed_form_by_quadrature():
    """The closed form c_l(k) = k^{l+1} e^{-k^2/4a} / (2a)^{l+3/2} of the SBT
    (Eq. (2)) of psi = r^{l+1} e^{-a r^2}, checked by adaptive quadrature."""
    for l in (0, 1, 3, 6):
        for a in (0.5, 1.7):
            for k in (0.3, 1.1, 2.5):
                f = lambda r: np.sqrt(2 / np.pi) * k * r * spherical_jn(l, k * r) * r ** (l + 1) * np.exp(-a * r * r)
                q, _ = integrate.quad(f, 0, 40, limit=400, epsabs=1e-14, epsrel=1e-12)
                ref = k ** (l + 1) * np.exp(-k * k / (4 * a)) / (2 * a) ** (l + 1.5)
                assert abs(q - ref) < 1e-10


def test_gaussian_dsbt_converges_as_dk2():
    """Fig. 1 / Sec. 3: b_n / sqrt(w_n) -> s_l c_l(k_n) with error ~ dk^2 (ratio
    ~4 per doubling of r_max at fixed dr); exact for l = 0; extra coefficients
    (n < n0_l) vanish for smooth input (Sec. 2.5)."""
    for l in (0, 1, 2, 3, 4):
        errs = []
        for rmax in (12.8, 25.6, 51.2):
            psi, n, k, wn, c = gaussian_case(l, rmax, 0.2, 1.0)
            b = oracle.forward(l, psi[None, :])[0]
            sel = (n >= oracle.n0(l)) & (k < 6)
            errs.append(np.abs(b[sel] / np.sqrt(wn[sel]) - s_l(l) * c[sel]).max())
            p = oracle.p_of(l)
            if oracle.n0(l) > p:
                assert np.abs(b[: oracle.n0(l) - p]).max() < 1e-12
        if l == 0:
            assert max(errs) < 1e-13
        else:
            assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs


def test_basis_functions_converge_to_riccati_bessel():
    """Fig. 2 / Sec. 3: columns of F^T T^T scaled by s_l sqrt(N/2) tend to
    chi_l(k r) = k r j_l(k r) at fixed k with error ~ dk^2."""
    dr = 0.2
    for l in (1, 2, 3):
        errs = []
        for rmax in (12.8, 25.6, 51.2):
            N = int(round(rmax / dr))
            dk = np.pi / rmax
            kk = 16 * np.pi / 12.8          # the same k on every grid
            n = int(round(kk / dk))
            p = oracle.p_of(l)
            e = np.zeros((1, N))
            e[0, n - p] = 1.0
            chi_t = s_l(l) * np.sqrt(N / 2) * oracle.inverse(l, e)[0]
            r = (np.arange(1, N + 1) - 0.5) * dr
            sel = r < 6.0
            ref = kk * r * spherical_jn(l, kk * r)
            errs.append(np.abs(chi_t[sel] - ref[sel]).max())
        assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, (l, errs)


# ------------------------------------------------------------ invariants

def test_norm_roundtrip_adjoint():
    """Eq. (22) b^T b = psi^T psi; inverse(forward(x)) = x; <Ax, y> = <x, A^T y>."""
    rng = np.random.default_rng(3)
    N = 96
    for l in (0, 1, 4, 9, 30):
        x = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
        y = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
        b = oracle.forward(l, x)
        assert abs(np.linalg.norm(b) - np.linalg.norm(x)) < 1e-13 * np.linalg.norm(x)
        assert np.abs(oracle.inverse(l, b) - x).max() < 1e-13
        lhs = np.vdot(y, oracle.forward(l, x))
        rhs = np.vdot(oracle.inverse(l, y), x)
        assert abs(lhs - rhs) < 1e-12


def test_sampled_rows_match_full():
    """The sampled helpers (used for large-N checks) equal the full transform."""
    rng = np.random.default_rng(4)
    N = 80
    x = rng.standard_normal((3, N))
    for l in (2, 7):
        rows = [0, 3, 41, 79]
        full = oracle.forward(l, x)
        assert np.abs(oracle.forward_rows(l, x, rows) - full[:, rows]).max() < 1e-14
        inv = oracle.inverse(l, full)
        assert np.abs(oracle.inverse_cols(l, full, rows) - inv[:, rows]).max() < 1e-14
