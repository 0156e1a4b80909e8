"""Writes the exact-rational fixtures in this folder.  Calls only oracle.exact
(exact Fraction arithmetic from the paper's explicit formulas); run it from the
repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402


def write_dlop():
    path = os.path.join(HERE, "dlop_exact.txt")
    with open(path, "w") as fh:
        fh.write("# Exact DLOP values P_l(x, M) from the explicit falling-factorial sum\n")
        fh.write("# (Sec. 2.3, Eq. (29) with l(l,j) the shifted-Legendre coefficients).\n")
        fh.write("# columns: l M x numerator denominator\n")
        for M in (8, 13, 21):
            for l in range(0, min(M, 10) + 1):
                for x in range(-1, M + 1):
                    v = exact.dlop(l, M, x)
                    fh.write(f"{l} {M} {x} {v.numerator} {v.denominator}\n")


def write_rows():
    path = os.path.join(HERE, "t_rows_exact.txt")
    with open(path, "w") as fh:
        fh.write("# Exact rational parts of the rows of T_l (Sec. 2.4 Eqs. (38)-(39) with\n")
        fh.write("# theta(0)=1/2; Sec. 2.5 Eq. (43) without alpha_n): entry T_nm =\n")
        fh.write("# a_nm sqrt(w_m) / sqrt(g_n), g_n = sum_m a_nm^2 w_m, w_m = 1 - delta_m0/2.\n")
        fh.write("# line 'row N l r g_num g_den' then N entries 'num/den' (r = n - p_l).\n")
        for N in (6, 9):
            for l in range(0, 8):
                if exact.n0(l) > N:
                    continue
                A = exact.rows_a(N, l)
                p = exact.p_of(l)
                for r, row in enumerate(A):
                    g = sum(row[t] * row[t] * exact.w(t + p) for t in range(N))
                    fh.write(f"row {N} {l} {r} {g.numerator} {g.denominator}\n")
                    fh.write(" ".join(f"{v.numerator}/{v.denominator}" for v in row) + "\n")


if __name__ == "__main__":
    write_dlop()
    write_rows()
