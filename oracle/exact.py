"""Exact rational arithmetic for tiny DSBT cases (test infrastructure only).

Everything here follows the paper's explicit formulas with ``fractions.Fraction``
so that the FP64/binary128 oracle can be pinned against values that carry no
rounding at all:

* DLOP by the explicit falling-factorial sum of Sec. 2.3 (Eq. (29)):
  P_l(i, M) = sum_j l(l, j) i^{falling j} / M^{falling j}, where l(l, j) are the
  coefficients of the shifted Legendre polynomial P_l(1 - 2x) = sum_j l(l, j) x^j,
  namely l(l, j) = (-1)^j C(l, j) C(l + j, j).  (This is a different formula
  from the oracle's three-term recurrence.)
* DDLOP, Eq. (34): P'_l(i, M) = 2 / (1 + P_l(-1, M-1)) [P_l(i, M-1) - P_l(i-1, M-1)].
* The rows of I - L (Eqs. (38)-(39), theta(0) = 1/2) and the extra rows of
  Eq. (43), split as entry = a_nm * sqrt(w_m) with a_nm rational, so that all
  inner products sum_m a_nm a_km w_m are exact rationals.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb


def falling(x: int, j: int) -> int:
    """x^{falling j} = x (x-1) ... (x-j+1)."""
    v = 1
    for t in range(j):
        v *= (x - t)
    return v


def legendre_shift_coeff(l: int, j: int) -> int:
    """l(l, j): P_l(1 - 2x) = sum_j l(l, j) x^j."""
    return (-1) ** j * comb(l, j) * comb(l + j, j)


@lru_cache(maxsize=None)
def dlop(l: int, M: int, x: int) -> Fraction:
    """P_l(x, M) by the explicit sum (defined for l <= M)."""
    if l > M:
        raise ValueError("DLOP of degree l exists only for l <= M")
    s = Fraction(0)
    for j in range(l + 1):
        s += Fraction(legendre_shift_coeff(l, j) * falling(x, j), falling(M, j))
    return s


def dlop_norm(l: int, M: int) -> Fraction:
    """N(l, M) = (M + l + 1)^{falling l+1} / ((2l + 1) M^{falling l}), Eq. (28)."""
    return Fraction(falling(M + l + 1, l + 1), (2 * l + 1) * falling(M, l))


def ddlop(l: int, M: int, i: int) -> Fraction:
    """P'_l(i, M), Eq. (34)."""
    pm1 = dlop(l, M - 1, -1)
    return Fraction(2) / (1 + pm1) * (dlop(l, M - 1, i) - dlop(l, M - 1, i - 1))


def w(m: int) -> Fraction:
    """Trapezoid weight 1 - delta_{m0}/2 (Eq. (20) without the dk factor)."""
    return Fraction(1, 2) if m == 0 else Fraction(1)


def p_of(l: int) -> int:
    return 1 if l % 2 == 0 else 0


def n0(l: int) -> int:
    return (l + 2) // 2


def rows_a(N: int, l: int):
    """Rational parts a[n-p][m-p] of the unnormalised rows of T_l.

    Regular rows (n >= n0): (I - L)_{nm} = a_nm sqrt(w_m) with
      a_nm = P'_l(n - m, 2n) for m < n,  a_nn = 1 + P'_l(0, 2n) / 2,  0 above.
    Extra rows (p <= n < n0): a_nm = P_{2n-p}(N_l - m, 2 N_l) (Eq. (43) without
    alpha_n).  Returns a list of lists of Fractions.
    """
    p = p_of(l)
    Nl = N + p - 1
    A = []
    for n in range(p, Nl + 1):
        row = []
        for m in range(p, Nl + 1):
            if n >= n0(l):
                if m < n:
                    v = ddlop(l, 2 * n, n - m)
                elif m == n:
                    v = 1 + ddlop(l, 2 * n, 0) / 2
                else:
                    v = Fraction(0)
            else:
                v = dlop(2 * n - p, 2 * Nl, Nl - m)
            row.append(v)
        A.append(row)
    return A


def gram(N: int, l: int):
    """Exact G[n][k] = sum_m a_nm a_km w_m over the rows of rows_a()."""
    p = p_of(l)
    A = rows_a(N, l)
    ws = [w(m) for m in range(p, N + p)]
    G = [[sum(ra[t] * rb[t] * ws[t] for t in range(N)) for rb in A] for ra in A]
    return G
