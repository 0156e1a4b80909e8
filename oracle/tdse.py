"""Split-operator TDSE oracle (test infrastructure only).

Follows the step sequence of Sec. 4.1 (Eq. (81)) for an axially symmetric state
(m = 0, N_phi = 1) with vector potential A = 0 (length gauge), so that the
plane-wave exponential in the middle of the step is the identity:

    psi_1 = exp(-i U tau/2) psi            (angular grid, U = V(r) + E r eta)
    c_1   = B Y psi_1                      (Y = P: grid -> l;  B = T_l F_l per l)
    c_2   = exp(-i K tau/2) c_1            (K = k~_n^2 / 2, Eq. (76), grid Eq. (65))
    c_3   = c_2                            (A = 0)
    c_4   = exp(-i K tau/2) c_3
    psi_4 = Y^T B^T c_4
    psi'  = exp(-i U tau/2) psi_4

The state is kept on the (r_i, eta_j) grid, psi[j][i] = Psi(r_i, eta_j) r_i
sqrt(dr w_j) (the DVR of Sec. 4.1).  F_l and T_l come from the FP64 oracle;
the Gauss-Legendre rule from numpy; P[l][j] = sqrt((2l+1)/2) P_l(eta_j) sqrt(w_j)
(orthonormal on the rule).  Matrices are applied with numpy matmul.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import eval_legendre, gammaln, lpmv

import oracle


def angular(L: int, m: int = 0):
    """(eta, w, P) of the L-point Gauss-Legendre rule.  m = 0: P[l][j] =
    sqrt((2l+1)/2) P_l(eta_j) sqrt(w_j), l < L (orthonormal on the rule).
    m != 0 (Sec. 4.1: associated Legendre functions orthonormalised on the
    quadrature): rows l = |m| .. |m|+L-1 of the normalised associated Legendre
    functions (no Condon-Shortley sign) times sqrt(w_j), orthonormalised in
    order of l (QR with a positive diagonal, i.e. Gram-Schmidt)."""
    eta, w = leggauss(L)
    if m == 0:
        P = np.array([np.sqrt((2 * l + 1) / 2.0) * eval_legendre(l, eta) * np.sqrt(w) for l in range(L)])
        return eta, w, P
    m = abs(m)
    rows = []
    for l in range(m, m + L):
        norm = np.sqrt((2 * l + 1) / 2.0 * np.exp(gammaln(l - m + 1) - gammaln(l + m + 1)))
        rows.append((-1) ** m * norm * lpmv(m, l, eta) * np.sqrt(w))
    A = np.array(rows)
    Q, R = np.linalg.qr(A.T)                  # A^T = Q R: rows of Q^T orthonormal, same span in order
    Q = Q * np.sign(np.diag(R))[None, :]
    return eta, w, Q.T


class Model:
    """kcorr=True: the kinetic energy of Eq. (76) uses the corrected momenta
    k_nl of Sec. 3 (oracle/kcorr.py) instead of k~_n.  V: optional radial
    potential on the grid (default the soft Coulomb -Z / sqrt(r^2 + a2))."""

    def __init__(self, N: int, r_max: float, L: int, tau: float, Z: float = 1.0, a2: float = 0.5,
                 kcorr: bool = False, V=None, m: int = 0):
        self.N, self.r_max, self.L, self.tau = N, r_max, L, tau
        self.dr = r_max / N
        self.r = (np.arange(1, N + 1) - 0.5) * self.dr
        self.V = -Z / np.sqrt(self.r ** 2 + a2) if V is None else np.asarray(V, dtype=np.float64)
        self.eta, self.w, self.P = angular(L, m)
        self.ls = [abs(m) + i for i in range(L)]          # angular momentum of each channel
        self.F = [oracle.F_matrix(N, l) for l in self.ls]
        self.T = [oracle.T_matrix(N, l) for l in self.ls]
        self.kt = []
        for l in self.ls:
            if kcorr:
                from oracle import kcorr as kc
                self.kt.append(kc.k_table(N, r_max, l))
                continue
            self.kt.append(oracle.k_tilde(N, r_max, l))

    # l representation <-> angular grid (Y and Y^T)
    def to_l(self, psi_eta):
        return self.P @ psi_eta

    def to_eta(self, c):
        return self.P.T @ c

    def potential_half(self, psi_eta, E, tau):
        U = self.V[None, :] + E * self.r[None, :] * self.eta[:, None]
        return np.exp(-0.5j * tau * U) * psi_eta

    def step(self, psi_eta, E, tau=None):
        tau = self.tau if tau is None else tau
        psi1 = self.potential_half(psi_eta, E, tau)
        c = self.to_l(psi1)
        c4 = np.empty_like(c)
        for l in range(self.L):
            b = self.T[l] @ (self.F[l] @ c[l])
            half = np.exp(-0.5j * (self.kt[l] ** 2 / 2.0) * tau)
            b = half * (half * b)
            c4[l] = self.F[l].T @ (self.T[l].T @ b)
        psi4 = self.to_eta(c4)
        return self.potential_half(psi4, E, tau)

    def step_velocity(self, psi_eta, E, A, tau=None):
        """Eq. (81) with the vector potential A along z: between the two kinetic
        half steps, phi = Ytilde^dagger c on the momentum grid k~_n = n dk
        (Ytilde[l][j] = i^l P[l][j]), phi *= exp(i A k~_n eta_j tau), c = Ytilde
        phi.  The paper's spherical-wave coefficients are s_l times this
        library's (sine/cosine sign convention, s_l = (-1)^ceil(l/2))."""
        tau = self.tau if tau is None else tau
        N, L = self.N, self.L
        psi1 = self.potential_half(psi_eta, E, tau)
        c = self.to_l(psi1)
        coef = np.zeros((L, N), dtype=complex)        # [l][n - 1], n = 1..N
        for i, l in enumerate(self.ls):
            b = self.T[i] @ (self.F[i] @ c[i])
            b = np.exp(-0.25j * self.kt[i] ** 2 * tau) * b
            s_l = (-1) ** ((l + 1) // 2)
            n = np.arange(N) + oracle.p_of(l)
            slot = np.where(n == 0, N, n) - 1
            coef[i, slot] = s_l * b
        kt = np.arange(1, N + 1) * np.pi / self.r_max
        il = np.array([1j ** l for l in self.ls])
        phi = (np.conj(il)[:, None] * self.P).T @ coef                  # [j][n]
        phi = np.exp(1j * A * kt[None, :] * self.eta[:, None] * tau) * phi
        coef = (il[:, None] * self.P) @ phi                              # [l][n]
        c4 = np.empty_like(c)
        for i, l in enumerate(self.ls):
            s_l = (-1) ** ((l + 1) // 2)
            n = np.arange(N) + oracle.p_of(l)
            slot = np.where(n == 0, N, n) - 1
            b = np.exp(-0.25j * self.kt[i] ** 2 * tau) * (s_l * coef[i, slot])
            c4[i] = self.F[i].T @ (self.T[i].T @ b)
        psi4 = self.to_eta(c4)
        return self.potential_half(psi4, E, tau)

    def run(self, psi_eta, E_samples, nsteps: int, hold: int):
        x = psi_eta.copy()
        for s in range(nsteps):
            x = self.step(x, E_samples[s // hold])
        return x

    def observable(self, psi_eta, r_cut: float) -> float:
        sel = self.r > r_cut
        return float(np.sum(np.abs(psi_eta[:, sel]) ** 2))

    def gaussian_l0(self):
        """Normalised l = 0 state r exp(-r^2/2) in the l representation."""
        c = np.zeros((self.L, self.N), dtype=np.complex128)
        f = self.r * np.exp(-0.5 * self.r ** 2) * np.sqrt(self.dr)
        c[0] = f / np.linalg.norm(f)
        return c
