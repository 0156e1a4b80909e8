"""Plans with corrected momenta (DSBT_PLAN_KCORR, Sec. 3 Eq. (kcorr)): the
momentum table against the oracle's zero search (a different algorithm: the
library follows the Riccati-Bessel phase, the oracle scans sign changes), and
the kinetic step with those momenta against the oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import kcorr
from paper_1509_07115_gb300 import dsbt, inputs


def test_kcorr_flag_needs_a_factor_set():
    lib = dsbt.load()
    h = ctypes.c_void_p()
    assert lib.dsbt_plan_create(256, 25.6, 4, dsbt.DSBT_PLAN_KCORR, None, ctypes.byref(h)) == -1
    assert lib.dsbt_plan_create(256, 25.6, 4, 1024 | dsbt.DSBT_PLAN_FP64, None, ctypes.byref(h)) == -1   # unknown bit


@pytest.mark.gpu
@pytest.mark.parametrize("N, r_max, lmax", [(2048, 204.8, 40), (4352, 435.2, 64), (768, 38.4, 12)])
def test_momentum_table_matches_oracle(lib, N, r_max, lmax):
    p = lib.Plan(N, r_max, lmax, tf32x3=False, kcorr=True)
    for l in sorted({0, 1, 2, 3, lmax // 2, lmax - 1, lmax}):
        ref = kcorr.k_table(N, r_max, l)
        assert np.abs(p.get_k(l) - ref).max() <= 1e-13 * ref.max(), l
    p.close()
    q = lib.Plan(512, 51.2, 5, tf32x3=False)
    for l in range(6):
        assert np.abs(q.get_k(l) - oracle.k_tilde(512, 51.2, l)).max() < 1e-13
    q.close()


@pytest.mark.gpu
def test_kinetic_with_corrected_momenta_matches_oracle(lib):
    N, r_max, lmax, tau = 512, 51.2, 9, 0.05
    counts = [2] * (lmax + 1)
    counts[5] = 3
    plan = lib.Plan(N, r_max, lmax, kcorr=True)
    x = inputs.gaussian_sum(41, N, r_max / N, counts)
    ref = np.empty_like(x)
    c0 = 0
    for l, c in enumerate(counts):
        k = kcorr.k_table(N, r_max, l)
        ref[c0:c0 + c] = oracle.inverse(l, oracle.forward(l, x[c0:c0 + c]) * np.exp(-0.5j * k * k * tau))
        c0 += c
    nrm = np.linalg.norm(x, axis=1)
    y64 = plan.kinetic_grouped(counts, torch.from_numpy(x).cuda(), tau).cpu().numpy()
    assert (np.abs(y64 - ref).max(axis=1) / nrm).max() < 1e-12
    y32 = plan.kinetic_grouped(counts, torch.from_numpy(x.astype(np.complex64)).cuda(), tau).cpu().numpy()
    assert (np.abs(y32 - ref).max(axis=1) / nrm).max() < 3e-6
    plan.close()
