"""Corrected momenta k_nl (Sec. 3, Eq. (kcorr)) -- test infrastructure only.

The paper corrects the momentum of DSBT coefficient n so that the spherical
Bessel function matches the basis function's boundary condition at r_max:
chi_l(k r_max) = 0 for even l, chi_l'(k r_max) = 0 for odd l, with
chi_l(x) = x j_l(x).  It does not say which root belongs to which n.  Reading
taken here: the basis function of index n behaves near r_max like
sin(k_n r - l pi/2) (even l) or its cosine partner (odd l), so the phase of
chi_l must advance by the same number of half-waves; counting zeros from x = 0,
coefficient n takes the m-th positive zero with m = n - floor(l/2).  That is
m >= 1 exactly for the regular rows n >= n0_l = ceil((l+1)/2); the completion
rows n < n0_l have no partner zero and keep the momentum they have without
the correction (oracle.k_tilde: the largest grid momentum k~_N).  For large m the zeros approach the paper's estimate
k_nl ~ k_n - l(l+1) dk^2 / (2 pi^2 k_n).

Method: sign changes of chi_l (or chi_l') on a uniform scan from x = 0 with a
step far below the zero spacing, each bracket refined by bisection; chi_l from
scipy.special.spherical_jn.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import spherical_jn

import oracle


def chi(l: int, x):
    return x * spherical_jn(l, x)


def chi_d(l: int, x):
    return spherical_jn(l, x) + x * spherical_jn(l, x, derivative=True)


def zeros(l: int, count: int, derivative: bool, h: float = 0.02) -> np.ndarray:
    """The first `count` positive zeros of chi_l (or chi_l') in increasing order."""
    f = (lambda x: chi_d(l, x)) if derivative else (lambda x: chi(l, x))
    xmax = (count + l / 2.0 + 2.0) * math.pi
    x = np.arange(1, int(xmax / h) + 2) * h
    v = f(x)
    idx = np.nonzero(v[:-1] * v[1:] < 0)[0][:count]
    if len(idx) < count:
        raise RuntimeError(f"found {len(idx)} of {count} zeros for l={l}")
    a, b = x[idx].copy(), x[idx + 1].copy()
    fa = f(a)
    for _ in range(64):
        m = 0.5 * (a + b)
        fm = f(m)
        left = fa * fm <= 0
        b = np.where(left, m, b)
        a = np.where(left, a, m)
        fa = np.where(left, fa, fm)
    return 0.5 * (a + b)


def k_table(N: int, r_max: float, l: int) -> np.ndarray:
    """Momentum of each storage index s = n - p_l (s = 0..N-1) for one l:
    corrected k_nl on the regular rows, k~_N on the completion rows."""
    p, n0 = oracle.p_of(l), oracle.n0(l)
    n = np.arange(N) + p
    k = oracle.k_tilde(N, r_max, l)
    half = l // 2
    reg = n >= n0
    m_last = int(n[-1]) - half
    if m_last >= 1:
        z = zeros(l, m_last, derivative=(l % 2 == 1))
        k[reg] = z[n[reg] - half - 1] / r_max
    return k
