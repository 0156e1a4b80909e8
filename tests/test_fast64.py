"""FP64 contractions in O(N l log N) work (DSBT_PLAN_FAST64, csrc/fast64.cu):
the kinetic step and the TDSE of a fast plan against the dense FP64 plan and
the oracle.  Interval moments reproduce T_l f and T_l^T b exactly up to
rounding (oracle/fast.py pins the scheme on the CPU)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1509_07115_gb300 import dsbt, inputs


def test_fast64_flag_rules():
    lib = dsbt.load()
    h = ctypes.c_void_p()
    assert lib.dsbt_plan_create(1024, 102.4, 4, dsbt.DSBT_PLAN_FAST64 | dsbt.DSBT_PLAN_TF32X3, None,
                                ctypes.byref(h)) == -1          # needs the FP64 factors
    assert lib.dsbt_plan_create(768, 76.8, 4, dsbt.DSBT_PLAN_FAST64 | dsbt.DSBT_PLAN_FP64, None,
                                ctypes.byref(h)) == -1          # N / 64 = 12, not a power of two


def rel(a, b, nrm):
    return (np.abs(a - b).max(axis=1) / nrm).max()


@pytest.mark.gpu
@pytest.mark.parametrize("kcorr", [False, True])
def test_fast_kinetic_matches_dense_and_oracle(lib, kcorr):
    N, r_max, lmax, tau = 1024, 102.4, 63, 0.05
    counts = [1] * (lmax + 1)
    for l in (0, 1, 2, 7, 30, 63):
        counts[l] = 3
    x = inputs.gaussian_sum(51, N, r_max / N, counts)
    nrm = np.linalg.norm(x, axis=1)
    fast = lib.Plan(N, r_max, lmax, tf32x3=False, kcorr=kcorr, fast64=True)
    y = fast.kinetic_grouped(counts, torch.from_numpy(x).cuda(), tau).cpu().numpy()
    fast.close()
    dense = lib.Plan(N, r_max, lmax, tf32x3=False, kcorr=kcorr)
    yd = dense.kinetic_grouped(counts, torch.from_numpy(x).cuda(), tau).cpu().numpy()
    dense.close()
    assert rel(y, yd, nrm) < 1e-12
    if not kcorr:   # the oracle on the low l groups (its binary128 factors are slow at high l)
        c0 = 0
        for l, c in enumerate(counts):
            if l <= 7:
                k = oracle.k_tilde(N, r_max, l)
                ref = oracle.inverse(l, oracle.forward(l, x[c0:c0 + c]) * np.exp(-0.5j * k * k * tau))
                assert rel(y[c0:c0 + c], ref, nrm[c0:c0 + c]) < 1e-12, l
            c0 += c


@pytest.mark.gpu
def test_fast_tdse_matches_dense(lib):
    N, r_max, L, tau = 2048, 204.8, 64, 0.05
    E = torch.from_numpy(inputs.tdse_field(7, 100)).cuda()
    r = (np.arange(N) + 0.5) * (r_max / N)
    c0 = np.zeros((L, N), dtype=np.complex128)
    f = r * np.exp(-0.5 * r * r) * np.sqrt(r_max / N)
    c0[0] = f / np.linalg.norm(f)
    out = []
    for fast in (True, False):
        plan = lib.Plan(N, r_max, L - 1, tf32x3=False, fast64=fast)
        td = lib.Tdse(plan, L, tau, Z=1.0, a2=0.5)
        psi = torch.from_numpy(c0).cuda()
        td.propagate(psi, E, 200, 2)
        out.append(psi.cpu().numpy())
        td.close()
        plan.close()
    assert np.abs(out[0] - out[1]).max() < 1e-11
