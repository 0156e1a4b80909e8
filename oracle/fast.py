"""A stable fast multiplication by T_l and T_l^T -- test infrastructure only
(the stable variant that the monomial scheme of Sec. 2.6 calls for).

Fact used (Sec. 2.4, Eqs. (38)-(42)): on a regular row n of T_l the entries
T_nm = alpha_n P'_l(n - m, 2n) sqrt(w_m), m < n, are a polynomial of degree
l - 1 in m (up to the weight sqrt(w_0) = 1/sqrt(2) of column m = 0).  So on any
interval I of columns left of the row, the row divided by sqrt(w_m) lies in
the K = l dimensional space of polynomials of degree < l on I's points.  Instead of monomials (whose
prefix sums cancel catastrophically, see oracle/prefix.py) each interval gets
an orthonormal basis Q_I of that space on its own integer points, so every
coefficient is a bounded projection:

  forward  b_r = sum_{c in near(r)} T_rc f_c + sum_{I in far(r)} beta_{r,I} . M_I,
           M_I = Q_I^T (sqrt(w) f)_I (moments), beta_{r,I} = Q_I^T (T_{r,I} / sqrt(w_I));
  inverse  f_c = (near part) + sqrt(w_c) [Q_I W_I]_c,  W_I = sum_{r: I in far(r)} beta_{r,I} b_r.

Columns are cut into leaf blocks of B points; far(r) is the dyadic
decomposition of the leaf blocks left of r's leaf (one interval per set bit of
the leaf index), near(r) the rest of r's own leaf.  Moments of a parent
interval come from its children's through K x K transfer matrices (the parent's
basis restricted to a child is a polynomial of degree < K there), and the
inverse pushes W down the same tree, so the work per line is
O(N K log(N/B) + N K^2 / B + N B) instead of N^2 / 2.  Completion rows
(n < n0_l) are applied densely.  Everything is FP64; the plan data comes from the FP64 oracle T_l.
"""
from __future__ import annotations

import numpy as np

import oracle


def _basis(length: int, K: int) -> np.ndarray:
    """Orthonormal basis [length][K] of polynomials of degree < K on the points
    0..length-1 (QR of a scaled Vandermonde matrix in Legendre form)."""
    x = (2.0 * np.arange(length) + 1.0) / length - 1.0
    V = np.polynomial.legendre.legvander(x, K - 1)
    Q, R = np.linalg.qr(V)
    return Q * np.sign(np.diag(R))[None, :]


class Plan:
    """right=True: the completion rows n < n0_l (polynomials of degree < l in m
    as well, Sec. 2.5) take the columns right of leaf 0 through the right
    intervals (j, 1) = [B 2^j, B 2^(j+1)) instead of densely (forward only), as
    the split-TF32 interval scheme does."""

    def __init__(self, N: int, l: int, B: int = 64, right: bool = False):
        if N % B or (N // B) & (N // B - 1):
            raise ValueError("N / B must be a power of two")
        self.N, self.l, self.B = N, l, B
        self.right = right
        self.T = oracle.T_matrix(N, l)
        self.ne = oracle.n0(l) - oracle.p_of(l)           # completion rows (storage 0..ne-1)
        self.sw = np.ones(N)                               # sqrt(w_m): 1/sqrt(2) at m = 0 (odd l)
        if l % 2 == 1:
            self.sw[0] = np.sqrt(0.5)
        self.K = l
        self.nleaf = N // B
        self.levels = max(1, (self.nleaf - 1).bit_length())
        K = self.K
        if K == 0:
            return
        self.Q = [_basis(B << j, K) for j in range(self.levels)]
        # transfer: Q_parent restricted to child h (0 left, 1 right) = Q_child @ A[j][h]
        self.A = []
        for j in range(1, self.levels):
            half = B << (j - 1)
            Qp, Qc = self.Q[j], self.Q[j - 1]
            self.A.append([Qc.T @ Qp[:half], Qc.T @ Qp[half:]])
        # completion rows on the right intervals (j, 1): moments there come from
        # the level bases directly (columns >= B carry weight 1)
        self.beta_right = {}
        if right:
            for r in range(self.ne):
                for j in range(self.levels):
                    lo, hi = B << j, B << (j + 1)
                    self.beta_right[(r, j)] = self.Q[j].T @ self.T[r, lo:hi]
        # beta[r][j] = Q^T T[r, I_j(r)] for every far interval of row r
        self.beta = {}
        for r in range(self.ne, N):
            J = r // B
            for j in range(self.levels):
                if (J >> j) & 1:
                    i = (J >> j) - 1
                    lo, hi = (i << j) * B, ((i + 1) << j) * B
                    row = self.T[r, lo:hi] / self.sw[lo:hi]
                    self.beta[(r, j)] = self.Q[j].T @ row

    def _far_intervals(self, r):
        J = r // self.B
        for j in range(self.levels):
            if (J >> j) & 1:
                yield j, (J >> j) - 1

    def forward(self, f: np.ndarray) -> np.ndarray:
        """b = T_l f for one line f (storage order)."""
        N, B, K = self.N, self.B, self.K
        T = self.T
        b = np.zeros(N)
        if self.right and K > 0:                                       # completion rows
            for r in range(self.ne):
                s = T[r, :B] @ f[:B]
                for j in range(self.levels):
                    lo, hi = B << j, B << (j + 1)
                    s += self.beta_right[(r, j)] @ (self.Q[j].T @ f[lo:hi])
                b[r] = s
        else:
            b[:self.ne] = T[:self.ne] @ f
        if K == 0:
            b[self.ne:] = np.diag(T)[self.ne:] * f[self.ne:]
            return b
        g = self.sw * f
        # moments, leaves then upwards
        M = [None] * self.levels
        M[0] = np.einsum("ik,ni->nk", self.Q[0], g.reshape(self.nleaf, B))
        for j in range(1, self.levels):
            prev = M[j - 1]
            A0, A1 = self.A[j - 1]
            M[j] = prev[0::2] @ A0 + prev[1::2] @ A1
        for r in range(self.ne, N):
            J = r // B
            near = slice(J * B, r + 1)
            s = T[r, near] @ f[near]
            for j, i in self._far_intervals(r):
                s += self.beta[(r, j)] @ M[j][i]
            b[r] += s
        return b

    def inverse(self, bvec: np.ndarray) -> np.ndarray:
        """f = T_l^T b for one line b (storage order)."""
        N, B, K = self.N, self.B, self.K
        T = self.T
        f = T[:self.ne].T @ bvec[:self.ne]                              # completion rows
        if K == 0:
            f[self.ne:] += np.diag(T)[self.ne:] * bvec[self.ne:]
            return f
        breg = bvec.copy()
        breg[:self.ne] = 0.0
        W = [np.zeros((self.nleaf >> j, K)) for j in range(self.levels)]
        for r in range(self.ne, N):
            J = r // B
            near = slice(J * B, r + 1)
            cols = np.arange(J * B, r + 1)
            f[cols] += T[r, near] * breg[r]
            for j, i in self._far_intervals(r):
                W[j][i] += self.beta[(r, j)] * breg[r]
        for j in range(self.levels - 1, 0, -1):                         # push W down the tree
            A0, A1 = self.A[j - 1]
            W[j - 1][0::2] += W[j] @ A0.T
            W[j - 1][1::2] += W[j] @ A1.T
        f += self.sw * np.einsum("ik,nk->ni", self.Q[0], W[0]).reshape(N)
        return f

    def work(self) -> dict:
        return work(self.N, self.l, self.B)


def work(N: int, l: int, B: int = 64) -> dict:
    """Multiply-adds per line of each part of the fast forward (the inverse is
    the same) and of the dense triangle, for comparison."""
    K = l
    nleaf = N // B
    levels = max(1, (nleaf - 1).bit_length())
    ne = oracle.n0(l) - oracle.p_of(l)
    far = sum(K * bin(r // B).count("1") for r in range(ne, N)) if K else 0
    moments = (N * K + sum((nleaf >> j) * 2 * K * K for j in range(1, levels))) if K else 0
    return {"near": sum(r % B + 1 for r in range(ne, N)), "far": far, "moments": moments,
            "completion": ne * N, "dense": N * (N + 1) // 2}
