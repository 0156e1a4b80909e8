"""The fast multiplication by T_l of Sec. 2.6 (monomial prefix sums,
oracle/prefix.py) against the dense T_l: exact in structure (it agrees to
rounding for small l) but its rounding error grows by orders of magnitude with
l, which is why the library's fast FP64 path uses orthonormal polynomial bases
on dyadic intervals instead (oracle/fast.py, DSBT_PLAN_FAST64).  Measured (random
f, max |b_fast - b| / |f|): N = 256: 3e-17 (l = 2), 1e-15 (l = 8), 1e-12
(l = 16); N = 1024: 6e-13 (l = 16), 1.4e-9 (l = 24), 1.2e-6 (l = 32)."""
import numpy as np

import oracle
from oracle import prefix


def err(N, l, seed=0):
    f = np.random.default_rng(seed).standard_normal(N)
    b = oracle.T_matrix(N, l) @ f
    fast = prefix.forward_rows(N, l, f)
    p = oracle.p_of(l)
    return max(abs(fast[n] - b[n - p]) for n in fast) / np.linalg.norm(f)


def test_prefix_scheme_exact_for_small_l_and_unstable_for_large_l():
    e2, e8, e16 = err(256, 2), err(256, 8), err(256, 16)
    assert e2 < 1e-15
    assert e8 < 1e-13
    assert e16 > 100 * e8 and e16 > 1e-13, (e8, e16)
