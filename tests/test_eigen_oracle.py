"""Pins of the bound-state oracle (oracle/eigen.py) against the energies the
paper prints for H (Tables 1 and 2, tests/golden/h_bound_states.txt).

The l > 0 states depend on the whole DSBT (T_l rows and completion rows, F_l,
the corrected momenta k_nl and the large momentum of the completion rows) and
must agree with the printed six digits.  The printed l = 0 energies come from
the paper's imaginary-time runs; the exact eigenvalues of the same Hamiltonian
differ from them by a few 1e-5 to 1e-4 (less for smaller dr), the size of the
split-step error of imaginary time with a step of ~0.01 (pinned below with the
split propagator's own levels).  The effective potential must bring the s
states several times closer to the exact energies.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import eigen

HERE = os.path.dirname(os.path.abspath(__file__))
R_MAX = 102.4
GRIDS = (512, 1024, 2048)   # dr = 0.2, 0.1, 0.05


def golden():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "h_bound_states.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, n, l, *E = line.split()
        rows[(int(t), int(n), int(l))] = [float(v) for v in E]
    return rows


def computed(N, table):
    r = eigen.grid(N, R_MAX)
    U = -1.0 / r if table == 1 else eigen.effective_potential(N, R_MAX)
    return {l: eigen.levels(N, R_MAX, l, U, 3 - l) for l in (0, 1, 2)}


@pytest.mark.parametrize("table", [1, 2])
@pytest.mark.parametrize("gi", [0, 1])
def test_printed_energies(table, gi):
    N = GRIDS[gi]
    lev = computed(N, table)
    g = golden()
    for (t, n, l), E in g.items():
        if t != table:
            continue
        e = lev[l][n - l - 1]
        if l > 0:
            tol = 1.5e-6 if table == 1 else 2.5e-6     # printed to 6 decimals
        else:
            tol = (1.2e-4, 2.0e-5)[gi]                 # imaginary-time split error of the print
        assert abs(e - E[gi]) < tol, (table, n, l, N, e, E[gi])
        assert abs(e - E[3]) <= abs(E[gi] - E[3]) + tol    # no farther from exact than the print


def test_l0_print_matches_split_step_levels():
    """The printed 1s energy at dr = 0.2 (-0.505927) lies below the exact
    eigenvalue (-0.505831) by the split-step shift of imaginary time: the split
    propagator's leading level crosses it for a step between 0.005 and 0.01."""
    N = 512
    U = -1.0 / eigen.grid(N, R_MAX)
    exact = eigen.levels(N, R_MAX, 0, U, 1)[0]
    printed = golden()[(1, 1, 0)][0]
    lo = eigen.split_levels(N, R_MAX, 0, U, 1, 0.005)[0]
    hi = eigen.split_levels(N, R_MAX, 0, U, 1, 0.01)[0]
    assert hi < printed < lo < exact


def test_effective_potential_improves_s_states():
    """Table 2's point: with u_Z the s-state energies move several times closer
    to the exact -1/(2 n^2) than with -1/r, at every dr; p and d states stay."""
    for N in GRIDS[:2]:
        coul, eff = computed(N, 1), computed(N, 2)
        for n in (1, 2, 3):
            exact = -0.5 / n ** 2
            assert abs(eff[0][n - 1] - exact) < abs(coul[0][n - 1] - exact) / 4, (N, n)
        for l in (1, 2):
            assert np.abs(eff[l] - coul[l]).max() < 3e-6
