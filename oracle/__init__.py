"""FP64 CPU oracle for the orthogonal discrete spherical Bessel transform.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the library path never does.  It
shares no code with the CUDA implementation.

The arithmetic lives in ``dsbt_oracle.c`` (plain C, FP64, IEEE binary128 for the
DLOP recurrence).  This module compiles it with gcc on first use and wraps it
with numpy.  Complex channels are handled as two real lines (F_l and T_l are
real), so every C routine works on real lines only.

Index conventions follow Sec. 2.2 of the paper: for angular momentum l the
momentum index is n = p_l .. N + p_l - 1 with p_l = [1 + (-1)^l] / 2, stored at
position n - p_l; radial samples psi_i = psi(r_i) sqrt(dr), r_i = (i - 1/2) dr.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsbt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liborcl.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FMA contraction so that
    x86-64 and aarch64 produce the same bits).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_dlop.restype = ctypes.c_double
            lib.orc_dlop.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long]
            lib.orc_dlop_norm.restype = ctypes.c_double
            lib.orc_dlop_norm.argtypes = [ctypes.c_int, ctypes.c_long]
            lib.orc_ddlop.restype = ctypes.c_double
            lib.orc_ddlop.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long]
            lib.orc_T_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _dp]
            lib.orc_T_matrix.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
            lib.orc_F_matrix.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
            lib.orc_forward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.orc_inverse.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.orc_apply.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


# ------------------------------------------------------------------ scalars

def dlop(l: int, M: int, x: int) -> float:
    """P_l(x, M), Sec. 2.3 Eq. (27) (binary128 recurrence, rounded)."""
    return _load().orc_dlop(int(l), int(M), int(x))


def dlop_norm(l: int, M: int) -> float:
    """N(l, M) of Eq. (28)."""
    return _load().orc_dlop_norm(int(l), int(M))


def ddlop(l: int, M: int, i: int) -> float:
    """P'_l(i, M) of Eq. (34)."""
    return _load().orc_ddlop(int(l), int(M), int(i))


def n0(l: int) -> int:
    """n_{0l} = ceil((l + 1) / 2), Sec. 2.4."""
    return (l + 2) // 2


def p_of(l: int) -> int:
    """p_l = [1 + (-1)^l] / 2, Eq. (17)."""
    return 1 if l % 2 == 0 else 0


# ------------------------------------------------------------------ matrices

def k_tilde(N: int, r_max: float, l: int) -> np.ndarray:
    """Momenta of the kinetic energy K = k^2/2 for storage index s = n - p_l
    (Eq. (65) and the remark after it): k~_n = n pi / r_max on the regular
    rows; the completion rows n < n0_l (Sec. 2.5; n = 0 of odd l among them)
    project onto non-regular high-frequency functions and take the largest
    grid momentum k~_N."""
    n = np.arange(N) + p_of(l)
    return np.where(n < n0(l), N, n) * (math.pi / r_max)


def T_matrix(N: int, l: int) -> np.ndarray:
    """Full T_l (Sec. 2.4-2.5), [N][N], entry (n - p_l, m - p_l)."""
    T = np.empty((N, N), dtype=np.float64)
    _check(_load().orc_T_matrix(int(N), int(l), _ptr(T)), "T_matrix")
    return T


def T_rows(N: int, l: int, rows) -> np.ndarray:
    """Selected rows (storage indices n - p_l) of T_l, [len(rows)][N]."""
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    out = np.empty((r.size, N), dtype=np.float64)
    _check(_load().orc_T_rows(int(N), int(l), int(r.size), r.ctypes.data_as(_ip), _ptr(out)),
           "T_rows")
    return out


def F_matrix(N: int, l: int) -> np.ndarray:
    """F_l of Eq. (16) (orthonormal DST-II for even l, DCT-II for odd l)."""
    F = np.empty((N, N), dtype=np.float64)
    _check(_load().orc_F_matrix(int(N), int(l), _ptr(F)), "F_matrix")
    return F


def apply(A: np.ndarray, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    """y = A x (or A^T x) on each real line of x ([lines][N]) by naive sums."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    N = A.shape[0]
    xs, cplx = _as_lines(x, N)
    y = np.empty_like(xs)
    _check(_load().orc_apply(int(N), _ptr(A), int(bool(transpose)), int(xs.shape[0]),
                             _ptr(xs), _ptr(y)), "apply")
    return _from_lines(y, cplx, x.shape)


# ------------------------------------------------------------------ transforms

def _as_lines(x: np.ndarray, N: int):
    x = np.asarray(x)
    if x.shape[-1] != N:
        raise ValueError("last axis must have length N")
    if np.iscomplexobj(x):
        z = np.ascontiguousarray(x.reshape(-1, N), dtype=np.complex128)
        lines = np.empty((2 * z.shape[0], N), dtype=np.float64)
        lines[0::2] = z.real
        lines[1::2] = z.imag
        return lines, True
    return np.ascontiguousarray(x.reshape(-1, N), dtype=np.float64), False


def _from_lines(lines: np.ndarray, cplx: bool, shape):
    if cplx:
        return (lines[0::2] + 1j * lines[1::2]).reshape(shape)
    return lines.reshape(shape)


def forward(l: int, psi: np.ndarray) -> np.ndarray:
    """b = T_l F_l psi for every channel (last axis = radial index, length N).
    Real or complex input; complex is transformed as two real lines."""
    N = np.asarray(psi).shape[-1]
    xs, cplx = _as_lines(psi, N)
    out = np.empty_like(xs)
    _check(_load().orc_forward(int(N), int(l), int(xs.shape[0]), _ptr(xs), _ptr(out)), "forward")
    return _from_lines(out, cplx, np.asarray(psi).shape)


def inverse(l: int, b: np.ndarray) -> np.ndarray:
    """psi = F_l^T T_l^T b (Eq. (25) with T^{-1} = T^T)."""
    N = np.asarray(b).shape[-1]
    xs, cplx = _as_lines(b, N)
    out = np.empty_like(xs)
    _check(_load().orc_inverse(int(N), int(l), int(xs.shape[0]), _ptr(xs), _ptr(out)), "inverse")
    return _from_lines(out, cplx, np.asarray(b).shape)


def forward_rows(l: int, psi: np.ndarray, rows) -> np.ndarray:
    """Sampled forward outputs: b[..., rows] for every channel, forming the
    full f = F_l psi but only the requested rows of T_l (large-N checks)."""
    N = np.asarray(psi).shape[-1]
    F = F_matrix(N, l)
    f = apply(F, psi)
    Tr = T_rows(N, l, rows)
    return f @ Tr.T


def inverse_cols(l: int, b: np.ndarray, cols) -> np.ndarray:
    """Sampled inverse outputs psi[..., cols]: f = T_l^T b in full (naive), then
    only the requested rows of F_l^T."""
    N = np.asarray(b).shape[-1]
    T = T_matrix(N, l)
    f = apply(T, b, transpose=True)
    F = F_matrix(N, l)
    return f @ F[:, np.asarray(cols)]
