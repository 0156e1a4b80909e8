"""Pins of the corrected-momentum oracle (oracle/kcorr.py, Sec. 3 Eq. (kcorr)).

Independent checks: for l = 0, 1, 2 the conditions chi_l(x) = 0 / chi_l'(x) = 0
reduce to elementary equations (sin x = 0; x cos x - sin x + x^2 sin x = 0;
(3 - x^2) sin x - 3 x cos x = 0) whose roots are found here by a separate scan
of those formulas; for large n the zeros approach the paper's estimate
k_nl ~ k_n - l(l+1) dk^2 / (2 pi^2 k_n) with an error falling like n^-3; the
completion rows take k~_N; corrected momenta increase with n, lie below k_n
and their spacing tends to dk.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import kcorr


def elementary_roots(g, count, h=1e-3):
    x = np.arange(1, int((count + 3) * math.pi / h)) * h
    v = g(x)
    idx = np.nonzero(v[:-1] * v[1:] < 0)[0][:count]
    a, b = x[idx], x[idx + 1]
    for _ in range(60):
        m = 0.5 * (a + b)
        left = g(a) * g(m) <= 0
        a, b = np.where(left, a, m), np.where(left, m, b)
    return 0.5 * (a + b)


@pytest.mark.parametrize("l, g", [
    (0, lambda x: np.sin(x)),
    (1, lambda x: x * np.cos(x) - np.sin(x) + x * x * np.sin(x)),
    (2, lambda x: (3.0 - x * x) * np.sin(x) - 3.0 * x * np.cos(x)),
])
def test_low_l_match_elementary_equations(l, g):
    N, r_max = 256, 25.6
    k = kcorr.k_table(N, r_max, l)
    n = np.arange(N) + oracle.p_of(l)
    reg = n >= oracle.n0(l)
    m = n[reg] - l // 2
    ref = elementary_roots(g, int(m.max()))[m - 1] / r_max
    assert np.abs(k[reg] - ref).max() < 1e-12 * ref.max()
    if l == 0:
        assert np.abs(k - n * math.pi / r_max).max() < 1e-13


@pytest.mark.parametrize("l", [3, 10, 31])
def test_large_n_approaches_paper_estimate(l):
    N, r_max = 4096, 409.6
    dk = math.pi / r_max
    k = kcorr.k_table(N, r_max, l)
    n = np.arange(N) + oracle.p_of(l)
    kn = np.where(n == 0, N, n) * dk
    est = kn - l * (l + 1) * dk * dk / (2 * math.pi ** 2 * kn)
    err = np.abs(k - est)
    i1, i2 = 20 * (l + 1), 40 * (l + 1)       # doubling n: error / 8
    ratio = err[i1] / err[i2]
    assert 6.0 < ratio < 10.0, ratio
    assert err[i2] < 1e-3 * (kn[i2] - est[i2])   # the estimate's correction itself is much larger


@pytest.mark.parametrize("l", [4, 5, 20, 63, 64])
def test_structure(l):
    N, r_max = 1024, 102.4
    dk = math.pi / r_max
    k = kcorr.k_table(N, r_max, l)
    n = np.arange(N) + oracle.p_of(l)
    kn = np.where(n == 0, N, n) * dk
    reg = n >= oracle.n0(l)
    assert np.all(k[~reg] == N * dk)                             # completion rows: k~_N
    assert np.all(k[reg] < kn[reg]) and np.all(np.diff(k[reg]) > 0)
    assert abs(np.diff(k[reg])[-1] - dk) < 1e-3 * dk              # spacing -> dk
