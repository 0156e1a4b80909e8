"""Exact solution of the 3-D harmonic oscillator in a uniform time-dependent
field (the benchmark of Sec. 4.3), projected on the DSBT-DVR state layout.

H = p^2/2 + r^2/2 + F(t) z.  The ground state stays a Gaussian displaced to the
classical path:  Psi = pi^{-3/4} exp(-(x^2 + y^2)/2 - (z - a)^2/2 + i p (z - a)
+ i (g - t)),  a' = p,  p' = -a - F,  g' = p^2/2 - a^2/2 - F a - 1/2,  all zero
at t = 0 (the x, y factors contribute exp(-i t/2) each).  In the velocity gauge
(A(t) = -A0 sin(omega t), F = dA/dt) the state is exp(i int A^2/2) exp(i A z)
times the length-gauge state.  In the state layout
of the propagator (l = 0..L-1, m = 0): psi_l(r_i) = sqrt(dr) r_i
sqrt(2 pi) int Psi(r_i, eta) Pbar_l(eta) d eta with Pbar_l = sqrt((2l+1)/2) P_l.
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.integrate import solve_ivp
from scipy.special import eval_legendre

A0 = 0.25


def vector_potential(t, omega):
    """A(t) = -A0 sin(omega t) of the velocity gauge (q E = -dA/dt)."""
    return -A0 * math.sin(omega * t)


def velocity_state(r, dr, L, T, omega):
    """Exact velocity-gauge state: H_v = p^2/2 - A p + r^2/2 (no A^2/2 term) gives
    psi_v = exp(i int_0^T A^2/2 dt) exp(i A(T) z) psi_length."""
    phase = 0.5 * A0 ** 2 * (T / 2 - math.sin(2 * omega * T) / (4 * omega))
    return state(r, dr, L, T, omega, kick=vector_potential(T, omega)) * np.exp(1j * phase)


def field(t, omega):
    """Coefficient F(t) of z in the Hamiltonian (the -qE(t) z of the coordinate
    gauge with qE = omega A0 cos(omega t))."""
    return -omega * A0 * math.cos(omega * t)


def classical(T, omega):
    def f(t, y):
        F = field(t, omega)
        return [y[1], -y[0] - F, 0.5 * y[1] ** 2 - 0.5 * y[0] ** 2 - F * y[0] - 0.5]
    s = solve_ivp(f, (0.0, T), [0.0, 0.0, 0.0], rtol=1e-12, atol=1e-14, method="DOP853")
    return s.y[:, -1]


def state(r, dr, L, T, omega, nquad=200, kick=0.0):
    """psi_l(r_i) of the exact solution at time T, array [L][N]; kick multiplies
    the state by exp(i kick z) (the velocity-gauge factor exp(i A(T) z))."""
    a, p, g = classical(T, omega) if T > 0 else (0.0, 0.0, 0.0)
    x, w = leggauss(nquad)
    Pb = np.array([np.sqrt((2 * l + 1) / 2.0) * eval_legendre(l, x) for l in range(L)])
    psi = np.pi ** -0.75 * np.exp(-(r[None, :] ** 2 + a * a) / 2 - 1j * p * a + 1j * (g - T)
                                 + (a + 1j * (p + kick)) * r[None, :] * x[:, None])
    return np.sqrt(dr) * r[None, :] * (np.sqrt(2 * np.pi) * (Pb * w) @ psi)


def state_on_grid(r, dr, eta, w, T, omega, m):
    """Exact length-gauge state at time T sampled on the DVR grid (eta_j, r_i):
    psi[j][i] = R(r_i, eta_j) r_i sqrt(dr w_j) sqrt(2 pi), where Psi = R e^{i m phi}.
    m = 0: the displaced ground state; m = 1: the displaced state
    pi^{-3/4} (x + i y) exp(-(x^2 + y^2)/2) exp(-(z - a)^2/2 + ...), whose x, y
    factor has energy 2 (phase exp(-2 i t))."""
    a, p, g = classical(T, omega) if T > 0 else (0.0, 0.0, 0.0)
    rr, ee = r[None, :], eta[:, None]
    rho2 = rr * rr * (1 - ee * ee)
    z = rr * ee
    Rm = np.pi ** -0.75 * np.exp(-rho2 / 2 - (z - a) ** 2 / 2 + 1j * p * (z - a) + 1j * (g - (1 + m) * T))
    if m == 1:
        Rm = Rm * rr * np.sqrt(1 - ee * ee)
    return Rm * rr * np.sqrt(dr * w[:, None]) * np.sqrt(2 * np.pi)
