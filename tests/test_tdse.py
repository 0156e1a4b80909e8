"""Split-operator TDSE through the DSBT and its adjoint.

CPU tests pin the TDSE oracle (oracle/tdse.py) to exact facts: the angular
transform is orthogonal and reproduces the cos(theta) coupling of the l basis,
the step is unitary and palindromic, and with V = 0, E = 0 it reduces to the
closed-form free evolution exp(-i k~^2 t / 2) in the DSBT basis.  GPU tests
compare the CUDA propagator with the oracle and check the adjoint gradient
against central finite differences (the paper gives no gradient, so finite
differences are its reference).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import tdse as otdse
from paper_1509_07115_gb300 import inputs

SMALL = dict(N=256, r_max=25.6, L=16, tau=0.05)


# ------------------------------------------------------------------ oracle pins

def test_angular_transform_orthogonal_and_cos_coupling():
    """P P^T = I on the Gauss-Legendre rule, and P diag(eta) P^T is the exact
    cos(theta) matrix of the normalised Legendre basis:
    <l+1|cos|l> = (l+1)/sqrt((2l+1)(2l+3)), zero elsewhere."""
    L = 12
    eta, w, P = otdse.angular(L)
    assert np.abs(P @ P.T - np.eye(L)).max() < 1e-14
    C = P @ np.diag(eta) @ P.T
    ref = np.zeros((L, L))
    for l in range(L - 1):
        ref[l, l + 1] = ref[l + 1, l] = (l + 1) / np.sqrt((2 * l + 1) * (2 * l + 3))
    assert np.abs(C - ref).max() < 1e-14


def test_oracle_step_unitary_and_palindromic():
    m = otdse.Model(128, 12.8, 6, 0.05)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((6, 128)) + 1j * rng.standard_normal((6, 128))
    y = m.step(x, 0.03)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    z = m.step(y, 0.03, tau=-0.05)      # U(-tau) = U(tau)^-1 for the symmetric splitting
    assert np.abs(z - x).max() < 1e-12


def test_oracle_free_evolution_closed_form():
    """V = 0, E = 0: S steps equal exp(-i k~^2 tau S / 2) in the DSBT basis."""
    m = otdse.Model(128, 12.8, 5, 0.05, Z=0.0)
    rng = np.random.default_rng(1)
    c0 = rng.standard_normal((5, 128)) + 1j * rng.standard_normal((5, 128))
    x = m.to_eta(c0)
    S = 7
    for _ in range(S):
        x = m.step(x, 0.0)
    c = m.to_l(x)
    for l in range(5):
        b = oracle.forward(l, c0[l])
        ref = oracle.inverse(l, b * np.exp(-0.5j * m.kt[l] ** 2 * 0.05 * S))
        assert np.abs(c[l] - ref).max() < 1e-12


# ------------------------------------------------------------------ GPU

def small_case(seed=3, nsteps=20, hold=2):
    m = otdse.Model(**SMALL)
    E = inputs.tdse_field(seed, nsamples=(nsteps + hold - 1) // hold)
    c0 = m.gaussian_l0()
    return m, E, c0, nsteps, hold


@pytest.mark.gpu
def test_gpu_tdse_matches_oracle(lib):
    m, E, c0, nsteps, hold = small_case()
    plan = lib.Plan(SMALL["N"], SMALL["r_max"], SMALL["L"] - 1, tf32x3=False)
    td = lib.Tdse(plan, SMALL["L"], SMALL["tau"])
    eta, w, P = td.angular()
    o, om = np.argsort(eta), np.argsort(m.eta)          # node order is a convention
    assert np.abs(eta[o] - m.eta[om]).max() < 1e-14 and np.abs(w[o] - m.w[om]).max() < 1e-14
    assert np.abs(P[:, o] - m.P[:, om]).max() < 1e-14
    psi = torch.from_numpy(c0).cuda()
    td.propagate(psi, torch.from_numpy(E), nsteps, hold)
    ref = m.to_l(m.run(m.to_eta(c0), E, nsteps, hold))
    assert np.abs(psi.cpu().numpy() - ref).max() < 1e-12
    td.close()
    plan.close()


@pytest.mark.gpu
def test_gpu_tdse_free_evolution_closed_form(lib):
    """Z = 0, E = 0: S steps of the propagator = one kinetic step of tau * S."""
    N, L, tau, S = 512, 8, 0.05, 30
    plan = lib.Plan(N, 51.2, L - 1, tf32x3=False)
    td = lib.Tdse(plan, L, tau, Z=0.0)
    x = inputs.gaussian_sum(4, N, 0.1, [1] * L)
    psi = torch.from_numpy(x).cuda()
    td.propagate(psi, torch.zeros(S, dtype=torch.float64), S, 1)
    ref = plan.kinetic_grouped([1] * L, torch.from_numpy(x).cuda(), tau * S)
    assert (psi - ref).abs().max().item() < 1e-12
    td.close()
    plan.close()


def full_case(lib):
    """m = 0, l = 0..63, N = 2048, dr = 0.1, 400 steps of 0.05, soft-Coulomb
    -1/sqrt(r^2 + 0.5), 200 field samples (sin^2 envelope, amplitude 0.05) held
    for 2 steps each, observable = norm beyond r = 50, checkpoint every 20."""
    N, L, tau = 2048, 64, 0.05
    plan = lib.Plan(N, 204.8, L - 1, tf32x3=False)
    td = lib.Tdse(plan, L, tau, Z=1.0, a2=0.5)
    c0 = np.zeros((L, N), dtype=np.complex128)
    r = (np.arange(N) + 0.5) * 0.1
    f = r * np.exp(-0.5 * r * r) * np.sqrt(0.1)
    c0[0] = f / np.linalg.norm(f)
    E = torch.from_numpy(inputs.tdse_field(7, 200)).cuda()
    return plan, td, torch.from_numpy(c0).cuda(), E


@pytest.mark.gpu
def test_gpu_tdse_unitary_and_reversible_full(lib):
    plan, td, psi0, E = full_case(lib)
    psi = psi0.clone()
    td.propagate(psi, E, 400, 2)
    drift = abs(torch.linalg.vector_norm(psi).item() - 1.0)
    assert drift < 1e-12, drift
    O = td.observable(psi, 50.0).item()
    assert 1e-6 < O < 0.5
    td.propagate(psi, E, 400, 2, backward=True)
    assert (psi - psi0).abs().max().item() < 1e-10
    td.close()
    plan.close()


@pytest.mark.gpu
def test_gpu_adjoint_matches_finite_differences_full(lib):
    plan, td, psi0, E = full_case(lib)
    O, g = td.gradient(psi0, E, 400, 2, 50.0, K=20)

    def O_of(Ev):
        psi = psi0.clone()
        td.propagate(psi, Ev, 400, 2)
        return td.observable(psi, 50.0).item()

    assert abs(O.item() - O_of(E)) < 1e-14
    gh = g.cpu().numpy()
    # O carries ~1e-13 relative rounding after 400 steps, so a larger step with
    # Richardson extrapolation (truncation O(h^4)) keeps the difference quotient
    # accurate to ~1e-7 relative
    h = 1e-4

    def central(j, hh):
        Ep, Em = E.clone(), E.clone()
        Ep[j] += hh
        Em[j] -= hh
        return (O_of(Ep) - O_of(Em)) / (2 * hh)

    for j in list(np.argsort(-np.abs(gh))[:3]) + [150]:
        fd = (4 * central(j, h / 2) - central(j, h)) / 3      # Richardson: O(h^4) truncation
        assert abs(fd - gh[j]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gh).max()), (j, fd, gh[j])
    # directional derivative along a random direction
    rng = np.random.default_rng(0)
    d = torch.from_numpy(rng.standard_normal(200)).cuda()
    fd = (O_of(E + h * d) - O_of(E - h * d)) / (2 * h)
    ad = float((g * d).sum().item())
    assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    td.close()
    plan.close()


@pytest.mark.gpu
def test_gpu_adjoint_matches_oracle_finite_differences_small(lib):
    m, E, c0, nsteps, hold = small_case(seed=5, nsteps=24, hold=2)
    plan = lib.Plan(SMALL["N"], SMALL["r_max"], SMALL["L"] - 1, tf32x3=False)
    td = lib.Tdse(plan, SMALL["L"], SMALL["tau"])
    r_cut = 3.0
    O, g = td.gradient(torch.from_numpy(c0).cuda(), torch.from_numpy(E), nsteps, hold, r_cut, K=5)
    x0 = m.to_eta(c0)
    O_ref = m.observable(m.run(x0, E, nsteps, hold), r_cut)
    assert abs(O.item() - O_ref) < 1e-13
    h = 1e-5
    gh = g.cpu().numpy()
    for j in (0, 5, 11):
        Ep, Em = E.copy(), E.copy()
        Ep[j] += h
        Em[j] -= h
        fd = (m.observable(m.run(x0, Ep, nsteps, hold), r_cut) - m.observable(m.run(x0, Em, nsteps, hold), r_cut)) / (2 * h)
        assert abs(fd - gh[j]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gh).max()), (j, fd, gh[j])
    td.close()
    plan.close()


@pytest.mark.gpu
def test_autograd_function_uses_adjoint(lib):
    m, E, c0, nsteps, hold = small_case(seed=6, nsteps=16, hold=2)
    plan = lib.Plan(SMALL["N"], SMALL["r_max"], SMALL["L"] - 1, tf32x3=False)
    td = lib.Tdse(plan, SMALL["L"], SMALL["tau"])
    psi0 = torch.from_numpy(c0).cuda()
    Et = torch.from_numpy(E).cuda().requires_grad_(True)
    O = lib.TdseObservable.apply(Et, td, psi0, nsteps, hold, 3.0, 4)
    O.backward()
    _, g = td.gradient(psi0, Et.detach(), nsteps, hold, 3.0, K=4)
    assert torch.allclose(Et.grad, g, rtol=0, atol=1e-15)
    td.close()
    plan.close()
