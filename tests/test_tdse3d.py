"""The all-m DSBT-DVR propagator on the GPU (dsbt_tdse3d_*, csrc/tdse3d.cu)
against the oracle (oracle/tdse3d.py), against the fixed-m propagator for a
field along z, and against the analytic 3-D oscillator driven along x (the
benchmark of Sec. 4.3 turned off the symmetry axis, so every m takes part)."""
import math

import numpy as np
import pytest
import torch

from oracle import tdse3d
import _oscillator as osc


@pytest.mark.gpu
def test_matches_oracle(lib):
    N, r_max, L, M, tau = 256, 25.6, 4, 2, 0.05
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    t = lib.Tdse3d(plan, L, M, tau)
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = -1.0 / np.sqrt(r ** 2 + 0.5)
    t.set_potential(V)
    m3 = tdse3d.Model3d(N, r_max, L, M, tau, V=V)
    assert t.channels == m3.channels
    rng = np.random.default_rng(7)
    psi = (rng.standard_normal((t.nchan, N)) + 1j * rng.standard_normal((t.nchan, N))) * 0.05
    F = rng.standard_normal((3, 3)) * 0.05
    ref = m3.run(psi, F, 6, hold=2)
    out = t.propagate(torch.from_numpy(psi).cuda(), torch.from_numpy(F), 6, hold=2).cpu().numpy()
    t.close()
    plan.close()
    assert np.abs(out - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.gpu
def test_field_along_z_equals_fixed_m_propagator(lib):
    N, r_max, L, M, tau = 256, 25.6, 5, 2, 0.05
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = -1.0 / np.sqrt(r ** 2 + 0.5)
    t3 = lib.Tdse3d(plan, L, M, tau)
    t3.set_potential(V)
    rng = np.random.default_rng(11)
    psi = (rng.standard_normal((t3.nchan, N)) + 1j * rng.standard_normal((t3.nchan, N))) * 0.05
    Ez = np.array([0.02, -0.03, 0.01])
    F = np.zeros((3, 3))
    F[:, 2] = Ez
    out = t3.propagate(torch.from_numpy(psi).cuda(), torch.from_numpy(F), 6, hold=2).cpu().numpy()
    for m in range(-M, M + 1):
        idx = [t3.channels.index((abs(m) + i, m)) for i in range(L)]
        tm = lib.Tdse(plan, L, tau, m=abs(m))
        tm.set_potential(V)
        x = torch.from_numpy(np.ascontiguousarray(psi[idx])).cuda()
        ref = tm.propagate(x, torch.from_numpy(Ez), 6, 2).cpu().numpy()
        tm.close()
        assert np.abs(out[idx] - ref).max() < 1e-12 * np.abs(ref).max(), m
    t3.close()
    plan.close()


def grid_state(m3, T, omega, axis, kick=0.0, phase=0.0):
    """Exact oscillator state (field along `axis`) as channel coefficients:
    Y^H of r Psi sqrt(dr w_j 2 pi / NM) on the (theta_j, phi_q) grid; kick
    multiplies Psi by exp(i kick s) (s the coordinate along the axis) and phase
    by exp(i phase) (the velocity-gauge factors)."""
    a, p, g = osc.classical(T, omega) if T > 0 else (0.0, 0.0, 0.0)
    st = np.sqrt(1 - m3.eta ** 2)
    n = {0: np.outer(st, np.cos(m3.phi)), 1: np.outer(st, np.sin(m3.phi)), 2: np.outer(m3.eta, np.ones(m3.NM))}[axis]
    s = n.reshape(-1)[:, None] * m3.r[None, :]                    # coordinate along the field
    rr = m3.r[None, :]
    Psi = np.pi ** -0.75 * np.exp(-(rr ** 2 - s ** 2) / 2 - (s - a) ** 2 / 2 + 1j * p * (s - a) + 1j * (g - T)
                                  + 1j * kick * s + 1j * phase)
    wq = np.repeat(m3.w, m3.NM) * (2 * np.pi / m3.NM)
    gr = Psi * rr * np.sqrt(m3.dr * wq)[:, None]
    return m3.Y.conj().T @ gr


@pytest.mark.gpu
def test_oscillator_along_x_matches_analytic(lib):
    """H = p^2/2 + r^2/2 + F(t) x: the ground state stays a Gaussian displaced
    along x.  The error matches the same run with the field along z (where only
    m = 0 takes part) and the paper's size at this r_max (Sec. 4.3)."""
    N, r_max, L, M, omega = 256, 12.8, 12, 6, 2.0
    tau, steps = 0.005, 628
    T = tau * steps
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    t3 = lib.Tdse3d(plan, L, M, tau)
    r = (np.arange(N) + 0.5) * (r_max / N)
    t3.set_potential(0.5 * r ** 2)
    m3 = tdse3d.Model3d(N, r_max, L, M, tau)    # Y and the grid only
    delta = {}
    for axis in (0, 2):
        c0 = grid_state(m3, 0.0, omega, axis)
        c0 = c0 / np.linalg.norm(c0)
        F = np.zeros((steps, 3))
        F[:, axis] = [osc.field((s + 0.5) * tau, omega) for s in range(steps)]
        out = t3.propagate(torch.from_numpy(c0).cuda(), torch.from_numpy(F), steps).cpu().numpy()
        ex = grid_state(m3, T, omega, axis)
        ex = ex / np.linalg.norm(ex)
        delta[axis] = abs(1 - np.vdot(ex, out))
    t3.close()
    plan.close()
    print(f"oscillator delta: field along x {delta[0]:.3e}, along z {delta[2]:.3e}")
    assert delta[0] < 1.2e-3, delta
    assert abs(delta[0] - delta[2]) < 0.05 * delta[2], delta


@pytest.mark.gpu
def test_fast64_plan_gives_the_same_steps(lib):
    """The all-m propagator over a DSBT_PLAN_FAST64 plan (O(N l log N) FP64
    contractions) equals the dense FP64 plan's steps."""
    N, r_max, L, M, tau = 1024, 102.4, 8, 3, 0.05
    rng = np.random.default_rng(13)
    F = rng.standard_normal((4, 3)) * 0.03
    out = []
    for fast in (False, True):
        plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False, fast64=fast)
        t3 = lib.Tdse3d(plan, L, M, tau)
        r = (np.arange(N) + 0.5) * (r_max / N)
        t3.set_potential(-1.0 / np.sqrt(r ** 2 + 0.5))
        psi = np.zeros((t3.nchan, N), dtype=complex)
        f = r * np.exp(-0.5 * r * r)
        psi[t3.channels.index((0, 0))] = f / np.linalg.norm(f)
        out.append(t3.propagate(torch.from_numpy(psi).cuda(), torch.from_numpy(F), 8, hold=2).cpu().numpy())
        t3.close()
        plan.close()
    assert np.abs(out[0] - out[1]).max() < 1e-12


@pytest.mark.gpu
def test_velocity_gauge_matches_oracle(lib):
    N, r_max, L, M, tau = 256, 25.6, 4, 2, 0.05
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    t = lib.Tdse3d(plan, L, M, tau)
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = 0.5 * r * r
    t.set_potential(V)
    m3 = tdse3d.Model3d(N, r_max, L, M, tau, V=V)
    rng = np.random.default_rng(21)
    psi = (rng.standard_normal((t.nchan, N)) + 1j * rng.standard_normal((t.nchan, N))) * 0.05
    A = rng.standard_normal((3, 3)) * 0.2
    F = rng.standard_normal((3, 3)) * 0.02
    ref = psi.copy()
    for s in range(6):
        ref = m3.step_velocity(ref, F[s // 2], A[s // 2])
    out = t.propagate_velocity(torch.from_numpy(psi).cuda(), torch.from_numpy(A), 6, hold=2,
                               F=torch.from_numpy(F)).cpu().numpy()
    t.close()
    plan.close()
    assert np.abs(out - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.gpu
def test_velocity_gauge_oscillator_along_x_matches_analytic(lib):
    """Velocity gauge, A(t) = -A0 sin(omega t) along x: the exact state is
    exp(i int A^2/2) exp(i A(T) x) times the length-gauge one (Sec. 4.3)."""
    N, r_max, L, M, omega = 256, 12.8, 12, 6, 2.0
    tau, steps = 0.005, 628
    T = tau * steps
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    t3 = lib.Tdse3d(plan, L, M, tau)
    r = (np.arange(N) + 0.5) * (r_max / N)
    t3.set_potential(0.5 * r ** 2)
    m3 = tdse3d.Model3d(N, r_max, L, M, tau)
    phase = 0.5 * osc.A0 ** 2 * (T / 2 - math.sin(2 * omega * T) / (4 * omega))
    delta = {}
    for axis in (0, 2):
        c0 = grid_state(m3, 0.0, omega, axis)
        c0 = c0 / np.linalg.norm(c0)
        A = np.zeros((steps, 3))
        A[:, axis] = [osc.vector_potential((s + 0.5) * tau, omega) for s in range(steps)]
        out = t3.propagate_velocity(torch.from_numpy(c0).cuda(), torch.from_numpy(A), steps).cpu().numpy()
        ex = grid_state(m3, T, omega, axis, kick=osc.vector_potential(T, omega), phase=phase)
        ex = ex / np.linalg.norm(ex)
        delta[axis] = abs(1 - np.vdot(ex, out))
    t3.close()
    plan.close()
    print(f"velocity-gauge oscillator delta: along x {delta[0]:.3e}, along z {delta[2]:.3e}")
    assert delta[0] < 6e-4, delta
    assert abs(delta[0] - delta[2]) < 0.05 * delta[2], delta
