"""Pins of the all-m DSBT-DVR oracle (oracle/tdse3d.py): the transform Y = P Phi
is unitary; a field along z couples no m, so the step equals the pinned fixed-m
oracle (oracle/tdse.py) for every m; with no field and no potential S steps are
the closed-form kinetic phase; and the physics is rotation invariant (an s state
in a field along x spreads exactly as in the same field along z)."""
import numpy as np
import pytest

import oracle
from oracle import tdse as tdse1
from oracle import tdse3d


def test_transform_is_unitary():
    m = tdse3d.Model3d(64, 6.4, 5, 3, 0.05)
    n = m.Y.shape[0]
    assert m.Y.shape == (n, n) == (5 * 7, len(m.channels))
    assert np.abs(m.Y.conj().T @ m.Y - np.eye(n)).max() < 1e-13
    assert np.abs(m.Y @ m.Y.conj().T - np.eye(n)).max() < 1e-13


def test_field_along_z_is_the_fixed_m_model():
    N, r_max, L, M, tau = 128, 12.8, 4, 2, 0.05
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = -1.0 / np.sqrt(r ** 2 + 0.5)
    m3 = tdse3d.Model3d(N, r_max, L, M, tau, V=V)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((len(m3.channels), N)) + 1j * rng.standard_normal((len(m3.channels), N))
    out = m3.step(psi, (0.0, 0.0, 0.03))
    for mm in range(-M, M + 1):
        fm = tdse1.Model(N, r_max, L, tau, V=V, m=mm)
        idx = [m3.index(abs(mm) + i, mm) for i in range(L)]
        ref = fm.to_l(fm.step(fm.to_eta(psi[idx]), 0.03))
        assert np.abs(out[idx] - ref).max() < 1e-12 * np.abs(ref).max(), mm


def test_free_steps_are_the_kinetic_phase():
    N, r_max, L, M, tau, S = 64, 6.4, 3, 1, 0.07, 4
    m3 = tdse3d.Model3d(N, r_max, L, M, tau)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((len(m3.channels), N)) + 0j
    out = m3.run(psi, [(0.0, 0.0, 0.0)], S, hold=S)
    for c, (l, _) in enumerate(m3.channels):
        b = oracle.T_matrix(N, l) @ (oracle.F_matrix(N, l) @ psi[c])
        b = np.exp(-0.5j * oracle.k_tilde(N, r_max, l) ** 2 * tau * S) * b
        ref = oracle.F_matrix(N, l).T @ (oracle.T_matrix(N, l).T @ b)
        assert np.abs(out[c] - ref).max() < 1e-12


def test_rotation_invariance_of_an_s_state():
    N, r_max, L, M, tau, S = 128, 12.8, 8, 6, 0.05, 20
    m3 = tdse3d.Model3d(N, r_max, L, M, tau)
    psi = np.zeros((len(m3.channels), N), dtype=complex)
    f = m3.r * np.exp(-0.5 * m3.r ** 2)
    psi[m3.index(0, 0)] = f / np.linalg.norm(f)
    ax = m3.run(psi, [(0.05, 0.0, 0.0)], S, hold=S)
    az = m3.run(psi, [(0.0, 0.0, 0.05)], S, hold=S)
    ay = m3.run(psi, [(0.0, 0.05, 0.0)], S, hold=S)
    dx, dy, dz = (np.sum(np.abs(a) ** 2, axis=0) for a in (ax, ay, az))
    assert np.abs(dx - dz).max() < 1e-9 and np.abs(dy - dz).max() < 1e-9
    assert np.abs(dz.sum() - 1.0) < 1e-12                      # unitary
    assert np.sum(np.abs(ax[[c for c, (l, m) in enumerate(m3.channels) if m != 0]]) ** 2) > 1e-6   # m mixing


def test_velocity_gauge_along_z_is_the_fixed_m_model():
    """A vector potential along z couples no m: every m block of the all-m
    velocity step equals the fixed-m oracle's velocity step."""
    N, r_max, L, M, tau = 128, 12.8, 4, 2, 0.05
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = 0.5 * r * r
    m3 = tdse3d.Model3d(N, r_max, L, M, tau, V=V)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal((len(m3.channels), N)) + 1j * rng.standard_normal((len(m3.channels), N))
    out = m3.step_velocity(psi, (0.0, 0.0, 0.01), (0.0, 0.0, 0.2))
    for mm in range(-M, M + 1):
        fm = tdse1.Model(N, r_max, L, tau, V=V, m=mm)
        idx = [m3.index(abs(mm) + i, mm) for i in range(L)]
        ref = fm.to_l(fm.step_velocity(fm.to_eta(psi[idx]), 0.01, 0.2))
        assert np.abs(out[idx] - ref).max() < 1e-12 * np.abs(ref).max(), mm


def test_velocity_gauge_rotation_invariance_and_unitarity():
    N, r_max, L, M, tau, S = 128, 12.8, 8, 6, 0.05, 10
    m3 = tdse3d.Model3d(N, r_max, L, M, tau)
    psi = np.zeros((len(m3.channels), N), dtype=complex)
    f = m3.r * np.exp(-0.5 * m3.r ** 2)
    psi[m3.index(0, 0)] = f / np.linalg.norm(f)
    out = {}
    for ax in (0, 2):
        A = [0.0, 0.0, 0.0]
        A[ax] = 0.3
        x = psi.copy()
        for _ in range(S):
            x = m3.step_velocity(x, (0.0, 0.0, 0.0), A)
        out[ax] = x
    dx, dz = (np.sum(np.abs(a) ** 2, axis=0) for a in (out[0], out[2]))
    assert abs(dz.sum() - 1.0) < 1e-12
    assert np.abs(dx - dz).max() < 1e-9
