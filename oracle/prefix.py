"""The fast multiplication by T_l of Sec. 2.6 (monomial prefix sums) --
test infrastructure only, kept to measure why the library contracts with the
dense T_l instead.

Regular rows n >= n0_l (Eq. (fast_b_f)): with the DDLOP expanded in powers of m,
P'_l(n - m, 2n) = -sum_nu xi_nu(n) m^nu (Eq. (DP_expan)),

    b_n = alpha_n f_n - alpha_n sum_nu xi_nu(n) s_nu(n),
    s_nu(n) = [nu = 0] f_0 / sqrt(2) + sum_{m=1}^{n-1} m^nu f_m + n^nu f_n / 2,

where the s_nu(n) are running (prefix) sums over m, O(l N) work in all.  The
coefficients xi_nu(n) are exact rationals here (the DDLOP from oracle/exact.py
at m = 0..l-1, then the exact inverse of that Vandermonde system), rounded to
FP64 once; the prefix sums and the combination run in FP64 as the paper
describes.  alpha_n comes from the FP64 oracle (the diagonal of T_l divided by
the rational diagonal entry 1 + P'_l(0, 2n)/2).  The cancellation between the
large terms xi_nu(n) s_nu(n) is what makes the scheme lose accuracy quickly
with l; completion rows and the rows n < l (too few points to fix the
polynomial from the row itself) are left to the dense oracle.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import oracle
from oracle import exact


def _inverse_vandermonde(l: int):
    """Exact inverse of V[m][nu] = m^nu, m, nu = 0..l-1 (as Fractions)."""
    V = [[Fraction(m) ** nu for nu in range(l)] for m in range(l)]
    n = l
    A = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(V)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        inv = 1 / A[c][c]
        A[c] = [v * inv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [row[n:] for row in A]


def xi(l: int, n: int, Vinv=None):
    """xi_nu(n), nu = 0..l-1, as Fractions (P'_l(n - m, 2n) = -sum xi_nu m^nu)."""
    Vinv = Vinv or _inverse_vandermonde(l)
    vals = [exact.ddlop(l, 2 * n, n - m) for m in range(l)]
    coef = [sum(Vinv[nu][m] * vals[m] for m in range(l)) for nu in range(l)]
    return [-c for c in coef]


def forward_rows(N: int, l: int, f: np.ndarray) -> dict:
    """b_n of the fast scheme for the regular rows n >= max(n0_l, l), FP64.
    f: storage-indexed real line (index m - p_l).  Returns {n: b_n}."""
    p = oracle.p_of(l)
    T = oracle.T_matrix(N, l)
    Vinv = _inverse_vandermonde(l) if l > 0 else None
    m = np.arange(p, N + p, dtype=np.float64)
    w = np.where(m == 0, np.sqrt(0.5), 1.0)
    out = {}
    # prefix sums S_nu(n) = sum_{m < n} sqrt(w_m) m^nu f_m (storage order = m order)
    pows = np.array([m ** nu for nu in range(max(l, 1))])          # [nu][m]
    terms = pows * (w * f)[None, :]
    S = np.cumsum(terms, axis=1) - terms                            # exclusive prefix sums
    for n in range(max(oracle.n0(l), l, p), N + p):
        s = n - p
        alpha = T[s, s] / float(1 + exact.ddlop(l, 2 * n, 0) / 2) if l > 0 else T[s, s]
        if l == 0:
            out[n] = alpha * f[s]
            continue
        xv = np.array([float(v) for v in xi(l, n, Vinv)])
        snu = S[:, s] + 0.5 * pows[:, s] * f[s]                     # s_nu(n) of the paper
        out[n] = alpha * f[s] - alpha * float(np.dot(xv, snu))
    return out
