"""Bound states of the DSBT-DVR Hamiltonian (Sec. 4.4) -- test infrastructure only.

For a spherical potential U(r) the l channels decouple.  In one channel the
approximate Hamiltonian of Eq. (H_DVR) is

    H_l = B_l^T diag(k_n^2 / 2) B_l + diag(U(r_i)),   B_l = T_l F_l,

with the kinetic momenta of the plan (oracle.k_tilde, or the corrected k_nl
of oracle/kcorr.py).  Its eigenvalues come from a dense symmetric eigensolver
(numpy.linalg.eigvalsh as a library step).  The paper reaches the same states
by imaginary-time evolution with the split propagator
S = exp(-U tau/2) B^T exp(-K tau) B exp(-U tau/2); `split_levels` returns the
levels -ln(lambda)/tau of S's leading eigenvalues, which that procedure
converges to for a step tau.

Effective potential (Eqs. (tilde_uZ), (uZ)): u~_Z makes the hydrogen-like
ground state phi_Z = r exp(-Z r) an exact eigenvector of the l = 0 Hamiltonian
with energy E_Z = -Z^2/2, i.e. u~_Z phi_Z = (E_Z - B^T K B) phi_Z.  The paper
prints the quotient with B^T (K - E_Z) B phi_Z in the numerator and no minus
sign; with that sign phi_Z is no eigenvector (the energies come out near -0.19
instead of -0.5), so the sign that makes phi_Z an eigenvector is taken.
u_Z = f u~_Z - (1 - f) Z / r with the mask f(r) = exp(-Z r).
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import kcorr as _kcorr


def grid(N: int, r_max: float) -> np.ndarray:
    return (np.arange(N) + 0.5) * (r_max / N)


def momenta(N: int, r_max: float, l: int, corrected: bool) -> np.ndarray:
    return _kcorr.k_table(N, r_max, l) if corrected else oracle.k_tilde(N, r_max, l)


def hamiltonian(N: int, r_max: float, l: int, U: np.ndarray, corrected: bool = True) -> np.ndarray:
    B = oracle.T_matrix(N, l) @ oracle.F_matrix(N, l)
    k = momenta(N, r_max, l, corrected)
    return B.T @ ((0.5 * k * k)[:, None] * B) + np.diag(U)


def levels(N: int, r_max: float, l: int, U: np.ndarray, count: int, corrected: bool = True) -> np.ndarray:
    """The `count` lowest eigenvalues of H_l."""
    return np.linalg.eigvalsh(hamiltonian(N, r_max, l, U, corrected))[:count]


def split_states(N: int, r_max: float, l: int, U: np.ndarray, count: int, tau: float,
                 corrected: bool = True):
    """Levels -ln(lambda_s)/tau of the `count` largest eigenvalues lambda_s of
    the imaginary-time split propagator S (symmetric), its eigenvectors
    (columns) and their energies <v|H_l|v>."""
    B = oracle.T_matrix(N, l) @ oracle.F_matrix(N, l)
    k = momenta(N, r_max, l, corrected)
    h = np.exp(-0.5 * tau * U)
    S = h[:, None] * (B.T @ (np.exp(-0.5 * tau * k * k)[:, None] * B)) * h[None, :]
    lam, V = np.linalg.eigh(0.5 * (S + S.T))
    lam, V = lam[::-1][:count], V[:, ::-1][:, :count]
    H = B.T @ ((0.5 * k * k)[:, None] * B) + np.diag(U)
    E = np.einsum("is,ij,js->s", V, H, V)
    return -np.log(lam) / tau, V, E


def split_levels(N: int, r_max: float, l: int, U: np.ndarray, count: int, tau: float,
                 corrected: bool = True) -> np.ndarray:
    return split_states(N, r_max, l, U, count, tau, corrected)[0]


def effective_potential(N: int, r_max: float, Z: float = 1.0) -> np.ndarray:
    r = grid(N, r_max)
    B = oracle.T_matrix(N, 0) @ oracle.F_matrix(N, 0)
    k = oracle.k_tilde(N, r_max, 0)
    phi = r * np.exp(-Z * r)
    EZ = -0.5 * Z * Z
    ut = -(B.T @ ((0.5 * k * k - EZ) * (B @ phi))) / phi
    f = np.exp(-Z * r)
    return f * ut - (1.0 - f) * Z / r
