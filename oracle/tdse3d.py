"""The full DSBT-DVR step with all m (Sec. 4.1) -- test infrastructure only.

Channels (l, m): m = -M .. M and, for each m, l = |m| .. |m| + L - 1, ordered
l-major (m ascending within l).  The angular grid is the L-point
Gauss-Legendre rule in eta = cos(theta) times NM = 2M + 1 angles
phi_q = 2 pi q / NM, and Y = P Phi (Sec. 4.1):

    Y[(j, q)][(l, m)] = Phi[m][q] P^|m|[l - |m|][j],   Phi[m][q] = exp(i m phi_q) / sqrt(NM),

with P^|m| the fixed-m rows of oracle/tdse.py (associated Legendre functions
without the Condon-Shortley sign, times sqrt(w_j), orthonormalised on the
rule), the library's convention, so that coefficients compare directly.
One step of length tau (A = 0, kinetic half steps merged), the state kept as
channel coefficients psi[c][i]:

    psi <- Q Kin Q psi,  Q = Y^H diag(exp(-i [V(r) + r F.n] tau/2)) Y,
    n = (sin theta cos phi, sin theta sin phi, cos theta),
    Kin: b = T_l F_l psi_c,  b *= exp(-i k~^2 tau/2),  psi_c = F_l^T T_l^T b,

with F_l, T_l and k~ from the FP64 oracle.  Y is built as one dense matrix and
applied with numpy matmul at every radial point.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import tdse as tdse1


class Model3d:
    def __init__(self, N: int, r_max: float, L: int, M: int, tau: float, V=None):
        self.N, self.r_max, self.L, self.M, self.tau = N, r_max, L, M, tau
        self.NM = 2 * M + 1
        self.dr = r_max / N
        self.r = (np.arange(N) + 0.5) * self.dr
        self.V = np.zeros(N) if V is None else np.asarray(V, dtype=np.float64)
        self.channels = [(l, m) for l in range(M + L) for m in range(-M, M + 1) if abs(m) <= l <= abs(m) + L - 1]
        self.eta, self.w, _ = tdse1.angular(L, 0)
        P = {am: tdse1.angular(L, am)[2] for am in range(M + 1)}   # already without the (-1)^m sign
        self.P = P
        phi = 2.0 * np.pi * np.arange(self.NM) / self.NM
        self.phi = phi
        nch = len(self.channels)
        Y = np.zeros((L * self.NM, nch), dtype=np.complex128)      # rows (j, q)
        for c, (l, m) in enumerate(self.channels):
            col = np.outer(P[abs(m)][l - abs(m)], np.exp(1j * m * phi) / np.sqrt(self.NM))   # [j][q]
            Y[:, c] = col.reshape(-1)
        self.Y = Y
        st = np.sqrt(np.maximum(0.0, 1.0 - self.eta ** 2))
        self.n = np.stack([np.outer(st, np.cos(phi)).reshape(-1), np.outer(st, np.sin(phi)).reshape(-1),
                           np.outer(self.eta, np.ones(self.NM)).reshape(-1)])   # [3][(j, q)]
        self.ls = sorted({l for l, _ in self.channels})
        self.F = {l: oracle.F_matrix(N, l) for l in self.ls}
        self.T = {l: oracle.T_matrix(N, l) for l in self.ls}
        self.kt = {l: oracle.k_tilde(N, r_max, l) for l in self.ls}

    def potential_half(self, psi, Fv, tau):
        g = self.Y @ psi                                             # [(j, q)][i]
        U = self.V[None, :] + (np.asarray(Fv, dtype=np.float64) @ self.n)[:, None] * self.r[None, :]
        g = np.exp(-0.5j * tau * U) * g
        return self.Y.conj().T @ g

    def kinetic(self, psi, tau):
        out = np.empty_like(psi)
        for c, (l, _) in enumerate(self.channels):
            b = self.T[l] @ (self.F[l] @ psi[c])
            b = np.exp(-0.5j * (self.kt[l] ** 2) * tau) * b
            out[c] = self.F[l].T @ (self.T[l].T @ b)
        return out

    def step(self, psi, Fv, tau=None):
        tau = self.tau if tau is None else tau
        x = self.potential_half(psi, Fv, tau)
        x = self.kinetic(x, tau)
        return self.potential_half(x, Fv, tau)

    def step_velocity(self, psi, Fv, Av, tau=None):
        """Eq. (81) with a vector potential A of any direction: between the two
        kinetic half steps, phi = Ytilde^H c on the momentum grid k~_n = n dk
        (Ytilde = Y with the factors i^l of the modified harmonics), phi *=
        exp(i k~_n (A . n) tau), c = Ytilde phi.  The spherical-wave
        coefficients are s_l = (-1)^ceil(l/2) times this library's, so the
        factor on c is (-i)^l s_l going in and i^l s_l coming out.  Momentum
        slot n holds storage n - 1 (even l) or n (odd l, slot N at storage 0)."""
        tau = self.tau if tau is None else tau
        N = self.N
        x = self.potential_half(psi, Fv, tau)
        coef = np.zeros((len(self.channels), N), dtype=complex)       # [ch][n - 1]
        slots = []
        for c, (l, _) in enumerate(self.channels):
            b = self.T[l] @ (self.F[l] @ x[c])
            b = np.exp(-0.25j * self.kt[l] ** 2 * tau) * b
            n = np.arange(N) + oracle.p_of(l)
            slot = np.where(n == 0, N, n) - 1
            slots.append(slot)
            s_l = (-1) ** ((l + 1) // 2)
            coef[c, slot] = (-1j) ** l * s_l * b
        kt = np.arange(1, N + 1) * np.pi / self.r_max
        phi = self.Y @ coef                                             # [(j, q)][n]
        phi = np.exp(1j * (np.asarray(Av, dtype=np.float64) @ self.n)[:, None] * kt[None, :] * tau) * phi
        coef = self.Y.conj().T @ phi
        out = np.empty_like(x)
        for c, (l, _) in enumerate(self.channels):
            s_l = (-1) ** ((l + 1) // 2)
            b = (1j) ** l * s_l * coef[c, slots[c]]
            b = np.exp(-0.25j * self.kt[l] ** 2 * tau) * b
            out[c] = self.F[l].T @ (self.T[l].T @ b)
        return self.potential_half(out, Fv, tau)

    def run(self, psi, F_samples, nsteps: int, hold: int = 1):
        x = psi.copy()
        for s in range(nsteps):
            x = self.step(x, F_samples[s // hold])
        return x

    def index(self, l: int, m: int) -> int:
        return self.channels.index((l, m))
