"""Adjoint gradient of the all-m DSBT-DVR propagator (dsbt_tdse3d_gradient):
dO/dF for O = sum over r > r_cut of |psi_S|^2 and the three components of every
field sample, against central finite differences of the GPU propagator and of
the oracle (oracle/tdse3d.py).  The paper has no gradient; the check is the
definition of the derivative."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import tdse3d
from paper_1509_07115_gb300 import dsbt


def test_gradient_rejects_bad_arguments_on_host():
    lib = dsbt.load()
    assert lib.dsbt_tdse3d_gradient_workspace_size(None, 10, 2) == 0
    assert lib.dsbt_tdse3d_gradient(None, None, None, 0, 0, 1, 0.0, 1, None, None, None, 0, None) == -1


def _setup(lib, N, r_max, L, M, tau, seed):
    plan = lib.Plan(N, r_max, M + L - 1, tf32x3=False)
    t = lib.Tdse3d(plan, L, M, tau)
    r = (np.arange(N) + 0.5) * (r_max / N)
    V = -1.0 / np.sqrt(r ** 2 + 0.5)
    t.set_potential(V)
    rng = np.random.default_rng(seed)
    psi = np.zeros((t.nchan, N), dtype=np.complex128)
    f = r * np.exp(-r * r / 18.0)
    psi[t.channels.index((0, 0))] = f
    psi += 0.02 * (rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)) * f
    psi /= np.linalg.norm(psi)
    return plan, t, r, V, psi, rng


def _observable(x, r, r_cut):
    return float((np.abs(x[:, r > r_cut]) ** 2).sum())


@pytest.mark.gpu
def test_gradient_matches_central_differences(lib):
    N, r_max, L, M, tau, nsteps, hold, r_cut = 256, 25.6, 5, 2, 0.05, 24, 2, 6.0
    plan, t, r, V, psi, rng = _setup(lib, N, r_max, L, M, tau, 3)
    F = 0.05 * rng.uniform(-1.0, 1.0, (nsteps // hold, 3))
    psi0 = torch.from_numpy(psi).cuda()
    O, g = t.gradient(psi0, F, nsteps, hold, r_cut, K=5)
    O, g = O.item(), g.cpu().numpy()
    x = t.propagate(psi0.clone(), F, nsteps, hold).cpu().numpy()
    assert abs(O - _observable(x, r, r_cut)) < 1e-13
    assert np.array_equal(psi0.cpu().numpy(), psi)          # psi0 is not modified
    h = 1e-4
    for (s, c) in [(0, 0), (3, 1), (5, 2), (7, 0), (11, 1), (11, 2)]:
        vals = []
        for sgn in (1, -1):
            Fp = F.copy()
            Fp[s, c] += sgn * h
            xp = t.propagate(psi0.clone(), Fp, nsteps, hold).cpu().numpy()
            vals.append(_observable(xp, r, r_cut))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[s, c] - fd) < 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (s, c, g[s, c], fd)
    t.close()
    plan.close()


@pytest.mark.gpu
def test_gradient_matches_oracle_differences(lib):
    """Tiny case: the oracle's propagator (explicit matrices, no GPU code)
    differentiated by central differences."""
    N, r_max, L, M, tau, nsteps, hold, r_cut = 256, 25.6, 3, 1, 0.05, 6, 2, 5.0
    plan, t, r, V, psi, rng = _setup(lib, N, r_max, L, M, tau, 5)
    F = 0.05 * rng.uniform(-1.0, 1.0, (nsteps // hold, 3))
    O, g = t.gradient(torch.from_numpy(psi).cuda(), F, nsteps, hold, r_cut, K=2)
    g = g.cpu().numpy()
    m3 = tdse3d.Model3d(N, r_max, L, M, tau, V=V)
    assert m3.channels == t.channels
    assert abs(O.item() - _observable(m3.run(psi, F, nsteps, hold=hold), r, r_cut)) < 1e-12
    h = 1e-4
    for s in range(nsteps // hold):
        for c in range(3):
            vals = []
            for sgn in (1, -1):
                Fp = F.copy()
                Fp[s, c] += sgn * h
                vals.append(_observable(m3.run(psi, Fp, nsteps, hold=hold), r, r_cut))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g[s, c] - fd) < 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (s, c, g[s, c], fd)
    t.close()
    plan.close()
