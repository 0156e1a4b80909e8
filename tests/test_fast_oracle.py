"""The stable fast multiplication by T_l and T_l^T (oracle/fast.py): every
row of T_l over an interval of columns left of it is a polynomial of degree
l - 1 (times sqrt(w_m)), so a hierarchy of intervals with orthonormal discrete
polynomial bases gives T_l f and T_l^T b with O(N l log N) work.  It must equal
the dense product to rounding for every l (odd l carries the m = 0 weight),
unlike the monomial scheme of Sec. 2.6 (tests/test_prefix_scheme.py)."""
import numpy as np
import pytest

from oracle import fast


@pytest.mark.parametrize("N, l, B", [(256, 0, 64), (256, 1, 64), (256, 2, 64), (256, 7, 64), (512, 10, 64),
                                     (512, 33, 64), (512, 63, 64), (256, 5, 32), (512, 20, 128)])
def test_fast_equals_dense(N, l, B):
    rng = np.random.default_rng(l)
    P = fast.Plan(N, l, B=B)
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


@pytest.mark.parametrize("l", [1, 2, 5, 12])
def test_row_left_of_diagonal_has_degree_l_minus_1(l):
    """The fact the scheme rests on (Eqs. (38)-(42)): on an interval of columns
    left of a regular row, T_nm / sqrt(w_m) is a polynomial of degree exactly
    l - 1 in m -- inside the span of the degree < l basis (residual at
    rounding), outside the span of degree < l - 1 (the top coefficient is
    small far from the row, but still orders of magnitude above rounding)."""
    import oracle
    N = 256
    T = oracle.T_matrix(N, l)
    sw = np.ones(N)
    if l % 2 == 1:
        sw[0] = np.sqrt(0.5)
    r = 200
    for lo, hi in ((0, 64), (64, 128), (128, 192)):
        row = T[r, lo:hi] / sw[lo:hi]
        Q = fast._basis(hi - lo, l)
        res = row - Q @ (Q.T @ row)
        assert np.abs(res).max() <= 1e-13 * np.abs(row).max(), (lo, np.abs(res).max())
        if l >= 2:
            Qs = fast._basis(hi - lo, l - 1)
            res_s = row - Qs @ (Qs.T @ row)
            assert np.abs(res_s).max() > 1e-11 * np.abs(row).max(), lo


@pytest.mark.parametrize("l", [1, 2, 5, 20, 63])
def test_completion_rows_are_polynomials_of_degree_below_l(l):
    """Sec. 2.5: the completion rows n < n0_l come from P_{2n-p}(N_l - m, 2N_l),
    a polynomial in m of degree 2n - p_l <= l - 1.  The split-TF32 interval
    scheme applies them right of leaf 0 through the same degree < l bases:
    on such an interval the row lies in the span of degree < l to rounding."""
    import oracle
    N = 1024
    T = oracle.T_matrix(N, l)
    ne = oracle.n0(l) - oracle.p_of(l)
    for r in range(ne):
        for lo, hi in ((128, 256), (256, 512), (512, 1024)):
            row = T[r, lo:hi]
            Q = fast._basis(hi - lo, l)
            res = row - Q @ (Q.T @ row)
            assert np.abs(res).max() <= 1e-12 * max(np.abs(row).max(), 1e-300), (r, lo)


@pytest.mark.parametrize("N, l", [(256, 1), (512, 6), (1024, 33), (1024, 63)])
def test_completion_rows_through_right_intervals(N, l):
    """The split-TF32 interval scheme's completion rows: leaf 0's columns densely,
    the columns right of it through the right intervals (j, 1) and the level
    bases.  Equals the dense product to rounding (leaves of 128)."""
    rng = np.random.default_rng(100 + l)
    P = fast.Plan(N, l, B=128, right=True)
    f = rng.standard_normal(N)
    b = P.T @ f
    tol = 1e-14 if l < 40 else 1e-12
    assert np.abs(P.forward(f) - b).max() <= tol * np.linalg.norm(f)
