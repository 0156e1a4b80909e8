"""The stable fast multiplication by T_l and T_l^T (oracle/fast.py): every
row of T_l over an interval of columns left of it is a polynomial of degree
l - 1 (times sqrt(w_m)), so a hierarchy of intervals with orthonormal discrete
polynomial bases gives T_l f and T_l^T b with O(N l log N) work.  It must equal
the dense product to rounding for every l (odd l carries the m = 0 weight),
unlike the monomial scheme of Sec. 2.6 (tests/test_prefix_scheme.py)."""
import numpy as np
import pytest

from oracle import fast


@pytest.mark.parametrize("N, l", [(256, 0), (256, 1), (256, 2), (256, 7), (512, 10), (512, 33), (512, 63)])
def test_fast_equals_dense(N, l):
    rng = np.random.default_rng(l)
    P = fast.Plan(N, l, B=64)
    f = rng.standard_normal(N)
    b = P.T @ f
    tol = 1e-14 if l < 40 else 1e-12
    assert np.abs(P.forward(f) - b).max() <= tol * np.linalg.norm(f)
    y = rng.standard_normal(N)
    assert np.abs(P.inverse(y) - P.T.T @ y).max() <= tol * np.linalg.norm(y)


def test_work_grows_like_l_n_log_n():
    """Multiply-adds per line against the dense triangle: at N = 4096 the fast
    scheme needs 4.5x fewer for l = 63 and 25x fewer for l = 8."""
    for l, gain in ((63, 4.0), (8, 20.0)):
        w = fast.work(4096, l)
        total = w["near"] + w["far"] + w["moments"] + w["completion"]
        assert w["dense"] / total > gain, (l, w)
