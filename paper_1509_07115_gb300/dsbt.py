"""ctypes binding of libdsbt.so (include/dsbt.h).  Argument marshalling only:
every step of the transform runs in the library's CUDA kernels.  There is no CPU
fallback: if the library cannot be loaded this module raises.

Tensors are torch tensors on the current CUDA device; the calls run on torch's
current stream.  Channel layout: last axis = radial index (length N), leading
axes flattened into channels; grouped calls take channels l-major.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

DSBT_OK = 0
DSBT_PLAN_FP64 = 1
DSBT_PLAN_TF32X3 = 2
DSBT_PLAN_KCORR = 4
DSBT_PLAN_FAST64 = 8
DSBT_PLAN_FAST_SPLIT = 16
DSBT_PLAN_FAST_TF32 = DSBT_PLAN_FAST_SPLIT   # earlier name of the same flag
DTYPES = {torch.float64: 1, torch.complex128: 2, torch.float32: 3, torch.complex64: 4}

_lib = None
_lock = threading.Lock()

_c_int_p = ctypes.POINTER(ctypes.c_int)


def load(auto_build: bool = True) -> ctypes.CDLL:
    """Load libdsbt.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if auto_build and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libdsbt.so not found at {_build.LIB}; run "
                               "`python -m paper_1509_07115_gb300.build`")
        lib = ctypes.CDLL(_build.LIB)
        vp, sz, i, d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
        lib.dsbt_plan_create.argtypes = [i, d, i, i, vp, ctypes.POINTER(vp)]
        lib.dsbt_plan_destroy.argtypes = [vp]
        lib.dsbt_plan_info.argtypes = [vp, _c_int_p, _c_int_p, _c_int_p, ctypes.POINTER(d)]
        lib.dsbt_plan_get_T.argtypes = [vp, i, vp, vp]
        lib.dsbt_plan_get_k.argtypes = [vp, i, vp]
        lib.dsbt_radial_states_workspace_size.restype = sz
        lib.dsbt_radial_states_workspace_size.argtypes = [vp, i]
        lib.dsbt_radial_states.argtypes = [vp, i, vp, i, d, i, vp, vp, vp, vp, sz, vp]
        lib.dsbt_workspace_size.argtypes = [vp, i, i]
        lib.dsbt_workspace_size.restype = sz
        for name in ("dsbt_forward", "dsbt_inverse"):
            getattr(lib, name).argtypes = [vp, i, i, i, vp, vp, vp, sz, vp]
        for name in ("dsbt_forward_grouped", "dsbt_inverse_grouped"):
            getattr(lib, name).argtypes = [vp, _c_int_p, i, vp, vp, vp, sz, vp]
        lib.dsbt_kinetic_grouped.argtypes = [vp, _c_int_p, i, d, vp, vp, vp, sz, vp]
        lib.dsbt_host_workspace_size.restype = sz
        lib.dsbt_host_workspace_size.argtypes = [vp, _c_int_p, i, i]
        for name in ("dsbt_forward_grouped_host", "dsbt_inverse_grouped_host"):
            getattr(lib, name).argtypes = [vp, _c_int_p, i, vp, vp, i, vp, sz, vp]
        lib.dsbt_kinetic_grouped_host.argtypes = [vp, _c_int_p, i, d, vp, vp, i, vp, sz, vp]
        lib.dsbt_device_status.argtypes = [vp, i, _c_int_p]
        lib.dsbt_plan_check.argtypes = [vp, ctypes.POINTER(d), vp]
        lib.dsbt_plan_set_spin_limit.argtypes = [vp, ctypes.c_uint]
        lib.dsbt_plan_set_fast_lag.argtypes = [vp, i]
        lib.dsbt_plan_perturb_T.argtypes = [vp, i, i, i, d, vp]
        lib.dsbt_last_error.restype = ctypes.c_char_p
        lib.dsbt_launch_count.restype = ctypes.c_longlong
        lib.dsbt_profile_enable.argtypes = [i]
        lib.dsbt_profile_read.argtypes = [i, _c_int_p, ctypes.POINTER(d)]
        lib.dsbt_kernel_name.argtypes = [i]
        lib.dsbt_kernel_name.restype = ctypes.c_char_p
        lib.dsbt_batch_create.argtypes = [i, _c_int_p, _c_int_p, _c_int_p, d, i, vp, ctypes.POINTER(vp)]
        lib.dsbt_batch_create_ex.argtypes = [i, _c_int_p, _c_int_p, _c_int_p, d, i, vp, ctypes.POINTER(vp)]
        lib.dsbt_batch_destroy.argtypes = [vp]
        lib.dsbt_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), _c_int_p, _c_int_p,
                                        ctypes.POINTER(ctypes.c_float)]
        lib.dsbt_batch_set_tiles.argtypes = [vp, i, i, vp]
        lib.dsbt_batch_tiles.argtypes = [i, _c_int_p, _c_int_p, _c_int_p, i, i, _c_int_p, _c_int_p,
                                         ctypes.POINTER(ctypes.c_longlong)]
        lib.dsbt_batch_forward.argtypes = [vp, vp, vp, vp]
        lib.dsbt_batch_kinetic.argtypes = [vp, d, vp, vp, vp]
        lib.dsbt_batch_capture_kinetic.argtypes = [vp, d, vp, vp, ctypes.POINTER(vp)]
        lib.dsbt_graph_launch.argtypes = [vp, vp]
        lib.dsbt_graph_destroy.argtypes = [vp]
        lib.dsbt_tdse_create.argtypes = [vp, i, d, d, d, ctypes.POINTER(vp)]
        lib.dsbt_tdse_destroy.argtypes = [vp]
        lib.dsbt_tdse_angular.argtypes = [vp, vp, vp, vp]
        lib.dsbt_tdse_set_potential.argtypes = [vp, vp, i]
        lib.dsbt_tdse_create_m.argtypes = [vp, i, i, d, d, d, ctypes.POINTER(vp)]
        lib.dsbt_tdse3d_create.argtypes = [vp, i, i, d, ctypes.POINTER(vp)]
        lib.dsbt_tdse3d_destroy.argtypes = [vp]
        lib.dsbt_tdse3d_channels.argtypes = [vp, _c_int_p, vp, vp]
        lib.dsbt_tdse3d_set_potential.argtypes = [vp, vp, i]
        lib.dsbt_tdse3d_workspace_size.argtypes = [vp]
        lib.dsbt_tdse3d_workspace_size.restype = sz
        lib.dsbt_tdse3d_propagate.argtypes = [vp, vp, vp, i, i, vp, sz, vp]
        lib.dsbt_tdse3d_propagate_velocity.argtypes = [vp, vp, vp, vp, i, i, vp, sz, vp]
        lib.dsbt_tdse3d_gradient_workspace_size.argtypes = [vp, i, i]
        lib.dsbt_tdse3d_gradient_workspace_size.restype = sz
        lib.dsbt_tdse3d_gradient.argtypes = [vp, vp, vp, i, i, i, d, i, vp, vp, vp, sz, vp]
        lib.dsbt_tdse_propagate_velocity.argtypes = [vp, vp, vp, vp, i, i, d, vp, sz, vp]
        lib.dsbt_tdse_workspace_size.argtypes = [vp, i, i]
        lib.dsbt_tdse_workspace_size.restype = sz
        lib.dsbt_tdse_propagate.argtypes = [vp, vp, vp, i, i, d, vp, sz, vp]
        lib.dsbt_tdse_observable.argtypes = [vp, vp, d, vp, vp]
        lib.dsbt_tdse_gradient.argtypes = [vp, vp, vp, i, i, i, d, i, vp, vp, vp, sz, vp]
        _lib = lib
        return lib


class DSBTError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != DSBT_OK:
        msg = load().dsbt_last_error().decode(errors="replace")
        raise DSBTError(f"{what} failed ({rc}): {msg}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A DSBT plan: T_l factors for l = 0..l_max on an N-point grid."""

    def __init__(self, N: int, r_max: float, l_max: int, fp64: bool = True, tf32x3: bool = True,
                 kcorr: bool = False, fast64: bool = False, fast_split: bool = False, fast_tf32: bool = False):
        lib = load()
        flags = (DSBT_PLAN_FP64 if fp64 else 0) | (DSBT_PLAN_TF32X3 if tf32x3 else 0) | \
            (DSBT_PLAN_KCORR if kcorr else 0) | (DSBT_PLAN_FAST64 if fast64 else 0) | \
            (DSBT_PLAN_FAST_SPLIT if (fast_split or fast_tf32) else 0)
        h = ctypes.c_void_p()
        _check(lib.dsbt_plan_create(int(N), float(r_max), int(l_max), flags, _stream(), ctypes.byref(h)),
               "dsbt_plan_create")
        self._h = h
        self.N, self.r_max, self.l_max, self.flags = int(N), float(r_max), int(l_max), flags
        self._ws = None

    # -------------------------------------------------------------- plumbing
    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dsbt_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        N, lm, fl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        err = ctypes.c_double()
        _check(load().dsbt_plan_info(self._h, ctypes.byref(N), ctypes.byref(lm), ctypes.byref(fl),
                                     ctypes.byref(err)), "dsbt_plan_info")
        return {"N": N.value, "l_max": lm.value, "flags": fl.value, "check_err": err.value}

    def workspace_bytes(self, total_channels: int, dtype: torch.dtype) -> int:
        return int(load().dsbt_workspace_size(self._h, int(total_channels), DTYPES[dtype]))

    def workspace(self, total_channels: int, dtype: torch.dtype, device=None) -> torch.Tensor:
        nb = self.workspace_bytes(total_channels, dtype)
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(max(nb, 256), dtype=torch.uint8,
                                   device=device or torch.cuda.current_device())
        return self._ws

    def _prep(self, x: torch.Tensor, out):
        if not x.is_cuda:
            raise ValueError("input must be a CUDA tensor")
        if x.shape[-1] != self.N:
            raise ValueError(f"last axis must be N={self.N}")
        if x.dtype not in DTYPES:
            raise ValueError(f"unsupported dtype {x.dtype}")
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        elif out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError("out must match the input's shape and dtype and be contiguous")
        return x, out

    # -------------------------------------------------------------- transforms
    def get_T(self, l: int) -> torch.Tensor:
        T = torch.empty((self.N, self.N), dtype=torch.float64, device="cuda")
        _check(load().dsbt_plan_get_T(self._h, int(l), ctypes.c_void_p(T.data_ptr()), _stream()),
               "dsbt_plan_get_T")
        return T

    def _single(self, name, l, x, out, workspace):
        x, out = self._prep(x, out)
        nchan = x.numel() // self.N
        ws = workspace if workspace is not None else self.workspace(nchan, x.dtype)
        _check(getattr(load(), name)(self._h, int(l), int(nchan), DTYPES[x.dtype],
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()), name)
        return out

    def forward(self, l: int, x: torch.Tensor, out=None, workspace=None) -> torch.Tensor:
        """b = T_l F_l x for every channel of x (dsbt_forward)."""
        return self._single("dsbt_forward", l, x, out, workspace)

    def inverse(self, l: int, b: torch.Tensor, out=None, workspace=None) -> torch.Tensor:
        """x = F_l^T T_l^T b (dsbt_inverse)."""
        return self._single("dsbt_inverse", l, b, out, workspace)

    def _counts(self, counts):
        c = list(int(v) for v in counts)
        if len(c) != self.l_max + 1:
            raise ValueError(f"counts needs l_max+1={self.l_max + 1} entries")
        return (ctypes.c_int * len(c))(*c), sum(c)

    def _grouped(self, name, counts, x, out, workspace, tau=None):
        x, out = self._prep(x, out)
        arr, total = self._counts(counts)
        if total * self.N != x.numel():
            raise ValueError("sum(counts) * N must equal the number of input elements")
        ws = workspace if workspace is not None else self.workspace(total, x.dtype)
        args = [self._h, arr, DTYPES[x.dtype]]
        if tau is not None:
            args.append(float(tau))
        args += [ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()]
        _check(getattr(load(), name)(*args), name)
        return out

    def forward_grouped(self, counts, x, out=None, workspace=None) -> torch.Tensor:
        return self._grouped("dsbt_forward_grouped", counts, x, out, workspace)

    def inverse_grouped(self, counts, b, out=None, workspace=None) -> torch.Tensor:
        return self._grouped("dsbt_inverse_grouped", counts, b, out, workspace)

    def kinetic_grouped(self, counts, x, tau: float, out=None, workspace=None) -> torch.Tensor:
        """F^T T^T exp(-i k~^2 tau / 2) T F x per l group (dsbt_kinetic_grouped)."""
        return self._grouped("dsbt_kinetic_grouped", counts, x, out, workspace, tau=tau)

    # ------------------------------------------- host-resident channels, streamed
    def host_workspace(self, counts, dtype: torch.dtype, chunks: int = 0) -> torch.Tensor:
        arr, _ = self._counts(counts)
        nb = int(load().dsbt_host_workspace_size(self._h, arr, DTYPES[dtype], int(chunks)))
        if nb == 0:
            raise DSBTError("dsbt_host_workspace_size failed: " + (load().dsbt_last_error() or b"").decode())
        return torch.empty(nb, dtype=torch.uint8, device=torch.cuda.current_device())

    def _grouped_host(self, name, counts, x, out, chunks, workspace, tau=None):
        if x.is_cuda or x.dtype not in DTYPES or not x.is_contiguous() or x.shape[-1] != self.N:
            raise ValueError("input must be a contiguous CPU tensor (pinned for overlap) with last axis N")
        arr, total = self._counts(counts)
        if total * self.N != x.numel():
            raise ValueError("sum(counts) * N must equal the number of input elements")
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        elif out.is_cuda or out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous CPU tensor matching the input")
        ws = workspace if workspace is not None else self.host_workspace(counts, x.dtype, chunks)
        args = [self._h, arr, DTYPES[x.dtype]]
        if tau is not None:
            args.append(float(tau))
        args += [ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(chunks),
                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()]
        _check(getattr(load(), name)(*args), name)
        return out

    def forward_grouped_host(self, counts, x, out=None, chunks: int = 0, workspace=None) -> torch.Tensor:
        """dsbt_forward_grouped on host tensors, streamed in chunks (asynchronous on
        the current stream: synchronise before reading `out`)."""
        return self._grouped_host("dsbt_forward_grouped_host", counts, x, out, chunks, workspace)

    def inverse_grouped_host(self, counts, b, out=None, chunks: int = 0, workspace=None) -> torch.Tensor:
        return self._grouped_host("dsbt_inverse_grouped_host", counts, b, out, chunks, workspace)

    def kinetic_grouped_host(self, counts, x, tau: float, out=None, chunks: int = 0, workspace=None):
        return self._grouped_host("dsbt_kinetic_grouped_host", counts, x, out, chunks, workspace, tau=tau)

    def get_k(self, l: int):
        """Momenta of the kinetic phase for angular momentum l (dsbt_plan_get_k)."""
        import numpy as np
        k = np.empty(self.N)
        _check(load().dsbt_plan_get_k(self._h, int(l), k.ctypes.data_as(ctypes.c_void_p)), "dsbt_plan_get_k")
        return k

    def radial_states(self, l: int, U, psi: torch.Tensor, tau: float, nsteps: int):
        """Imaginary-time bound states of channel l (dsbt_radial_states): psi is a
        float64 CUDA tensor [nstates][N] (start guess, overwritten with the
        states); returns (levels of the split propagator, energies <H>)."""
        import numpy as np
        if psi.dtype != torch.float64 or not psi.is_cuda or psi.dim() != 2 or psi.shape[1] != self.N \
                or not psi.is_contiguous():
            raise ValueError("psi must be a contiguous float64 CUDA tensor [nstates][N]")
        ns = psi.shape[0]
        Ud = torch.as_tensor(np.asarray(U, dtype=np.float64)).to("cuda").contiguous()
        nb = int(load().dsbt_radial_states_workspace_size(self._h, ns))
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device="cuda")
        lev, en = np.empty(ns), np.empty(ns)
        _check(load().dsbt_radial_states(self._h, int(l), _ptr(Ud), ns, float(tau), int(nsteps), _ptr(psi),
                                         lev.ctypes.data_as(ctypes.c_void_p), en.ctypes.data_as(ctypes.c_void_p),
                                         _ptr(ws), ws.numel(), _stream()), "dsbt_radial_states")
        return lev, en

    def check(self) -> float:
        """Re-run the orthogonality probe on the FP64 factors; raises
        DSBTError (code -3) when max |T^T T x - x| exceeds 1e-12."""
        err = ctypes.c_double()
        _check(load().dsbt_plan_check(self._h, ctypes.byref(err), _stream()), "dsbt_plan_check")
        return err.value

    def set_spin_limit(self, polls: int):
        """Testing hook: polls of each bounded device-side wait (0 = default)."""
        _check(load().dsbt_plan_set_spin_limit(self._h, int(polls)), "dsbt_plan_set_spin_limit")

    def set_fast_lag(self, lag: int):
        """Tile order of the interval-scheme contraction: units between a
        unit's moment (weight) tiles and its row tiles (>= 1; results do not
        depend on it)."""
        _check(load().dsbt_plan_set_fast_lag(self._h, int(lag)), "dsbt_plan_set_fast_lag")

    def perturb_T(self, l: int, row: int, col: int, delta: float):
        """Testing hook: add delta to one entry of the FP64 T_l."""
        _check(load().dsbt_plan_perturb_T(self._h, int(l), int(row), int(col), float(delta), _stream()),
               "dsbt_plan_perturb_T")

    def device_status(self, reset: bool = True) -> int:
        s = ctypes.c_int()
        _check(load().dsbt_device_status(self._h, int(bool(reset)), ctypes.byref(s)), "dsbt_device_status")
        return s.value


# ------------------------------------------------------------------ tracing

def launch_count() -> int:
    """Kernel launches issued by the library in this process."""
    return int(load().dsbt_launch_count())


def profile_enable(on: bool = True):
    """Start (and clear) or stop per-kernel CUDA-event timing in the library."""
    _check(load().dsbt_profile_enable(int(bool(on))), "dsbt_profile_enable")


def profile_read() -> dict:
    """{kernel name: (launches, total device ms)} of the recorded launches."""
    lib = load()
    out = {}
    k = 0
    while True:
        name = lib.dsbt_kernel_name(k)
        if name is None:
            break
        n, ms = ctypes.c_int(), ctypes.c_double()
        _check(lib.dsbt_profile_read(k, ctypes.byref(n), ctypes.byref(ms)), "dsbt_profile_read")
        if n.value:
            out[name.decode()] = (n.value, ms.value)
        k += 1
    return out


# ------------------------------------------------------------------ batch of uneven transforms

def batch_tiles(transforms, order: str, bn_cap: int) -> dict:
    """Host-only tile planning of a batch (dsbt_batch_tiles): forward and
    inverse tile counts and the forward B-operand lines, without a device."""
    Ns = [int(t[0]) for t in transforms]
    lms = [int(t[1]) for t in transforms]
    cnt = [int(v) for t in transforms for v in t[2]]
    arr = lambda v: (ctypes.c_int * len(v))(*v)
    f, i, sl = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(load().dsbt_batch_tiles(len(Ns), arr(Ns), arr(lms), arr(cnt), Batch.TILE_ORDERS.index(order),
                                   int(bn_cap), ctypes.byref(f), ctypes.byref(i), ctypes.byref(sl)),
           "dsbt_batch_tiles")
    return {"forward": f.value, "inverse": i.value, "seg_lines": sl.value}


class Batch:
    """Uneven transforms sharing one factor set (dsbt_batch_* in include/dsbt.h).
    transforms: list of (N_t, l_max_t, counts_t) with counts_t[l] channels of l.
    Batch arrays: complex64 CUDA tensors of total_elems elements, transforms back
    to back, each [sum(counts_t)][N_t] l-major."""

    def __init__(self, transforms, dr: float, autotune: bool = True, scheme: str = "dense"):
        """scheme: "dense" (shared split-TF32 factors, one persistent launch per
        direction, tile order and width autotuned when autotune) or "interval"
        (one interval-scheme plan per distinct grid, DSBT_BATCH_INTERVAL)."""
        if scheme not in ("dense", "interval"):
            raise ValueError("scheme is 'dense' or 'interval'")
        Ns = [int(t[0]) for t in transforms]
        lms = [int(t[1]) for t in transforms]
        cnt = []
        for (N, lm, c) in transforms:
            if len(c) != lm + 1:
                raise ValueError("counts_t needs l_max_t + 1 entries")
            cnt += [int(v) for v in c]
        arr = lambda v: (ctypes.c_int * len(v))(*v)
        h = ctypes.c_void_p()
        flags = (1 if (autotune and scheme == "dense") else 0) | (2 if scheme == "interval" else 0)
        _check(load().dsbt_batch_create_ex(len(Ns), arr(Ns), arr(lms), arr(cnt), float(dr), flags,
                                           _stream(), ctypes.byref(h)), "dsbt_batch_create")
        self.scheme = scheme
        self._h = h
        self.transforms = [(Ns[k], lms[k], list(transforms[k][2])) for k in range(len(Ns))]
        self.dr = float(dr)
        self._graphs = []

    def close(self):
        for g in self._graphs:
            load().dsbt_graph_destroy(g)
        self._graphs = []
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dsbt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        n, o, b = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 12)()
        _check(load().dsbt_batch_info(self._h, ctypes.byref(n), ctypes.byref(o), ctypes.byref(b), ms),
               "dsbt_batch_info")
        names = self.TILE_ORDERS
        if o.value < 0:   # interval scheme: no tile list
            return {"total_elems": n.value, "order": None, "bn_cap": 0, "tune_ms": {}}
        return {"total_elems": n.value, "order": names[o.value], "bn_cap": b.value,
                "tune_ms": {f"{names[k // 3]}/{[128, 192, 256][k % 3]}": ms[k] for k in range(12)}}

    TILE_ORDERS = ("transform-major", "l-major", "l-major/row-interleaved", "l-major/packed")

    def set_tiles(self, order: str, bn_cap: int):
        """Pin the contraction's tile order (one of TILE_ORDERS) and width."""
        _check(load().dsbt_batch_set_tiles(self._h, self.TILE_ORDERS.index(order), int(bn_cap), _stream()),
               "dsbt_batch_set_tiles")

    def offsets(self):
        """Complex-element offset of each transform in a batch array."""
        off, out = 0, []
        for (N, lm, c) in self.transforms:
            out.append(off)
            off += sum(c) * N
        return out

    def _check_arr(self, x):
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("batch arrays are contiguous complex64 CUDA tensors")
        if x.numel() != self.info()["total_elems"]:
            raise ValueError("batch array has the wrong number of elements")

    def forward(self, x, out=None):
        self._check_arr(x)
        out = torch.empty_like(x) if out is None else out
        _check(load().dsbt_batch_forward(self._h, _ptr(x), _ptr(out), _stream()), "dsbt_batch_forward")
        return out

    def kinetic(self, x, tau: float, out=None):
        self._check_arr(x)
        out = torch.empty_like(x) if out is None else out
        _check(load().dsbt_batch_kinetic(self._h, float(tau), _ptr(x), _ptr(out), _stream()), "dsbt_batch_kinetic")
        return out

    def capture_kinetic(self, x, tau: float, out):
        """CUDA graph of kinetic(x, tau, out); returns a handle for launch_graph."""
        self._check_arr(x)
        g = ctypes.c_void_p()
        _check(load().dsbt_batch_capture_kinetic(self._h, float(tau), _ptr(x), _ptr(out), ctypes.byref(g)),
               "dsbt_batch_capture_kinetic")
        self._graphs.append(g)
        return g

    @staticmethod
    def launch_graph(g):
        _check(load().dsbt_graph_launch(g, _stream()), "dsbt_graph_launch")


# ------------------------------------------------------------------ TDSE

class Tdse3d:
    """The full DSBT-DVR step with all m (dsbt_tdse3d_* in include/dsbt.h).
    State: complex128 CUDA tensor [nchan][N], channels l-major; ``channels``
    gives (l, m) per row.  Field samples F: [nsamples][3] (x, y, z)."""

    def __init__(self, plan: Plan, L: int, M: int, tau: float):
        import numpy as np
        h = ctypes.c_void_p()
        _check(load().dsbt_tdse3d_create(plan.handle, int(L), int(M), float(tau), ctypes.byref(h)),
               "dsbt_tdse3d_create")
        self._h, self.plan, self.L, self.M, self.N, self.tau = h, plan, int(L), int(M), plan.N, float(tau)
        n = ctypes.c_int()
        _check(load().dsbt_tdse3d_channels(h, ctypes.byref(n), None, None), "dsbt_tdse3d_channels")
        ls = np.empty(n.value, dtype=np.int32)
        ms = np.empty(n.value, dtype=np.int32)
        _check(load().dsbt_tdse3d_channels(h, ctypes.byref(n), ls.ctypes.data_as(ctypes.c_void_p),
                                           ms.ctypes.data_as(ctypes.c_void_p)), "dsbt_tdse3d_channels")
        self.nchan = n.value
        self.channels = list(zip(ls.tolist(), ms.tolist()))
        self._ws = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dsbt_tdse3d_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_potential(self, V):
        import numpy as np
        V = np.ascontiguousarray(V, dtype=np.float64)
        _check(load().dsbt_tdse3d_set_potential(self._h, V.ctypes.data_as(ctypes.c_void_p), int(V.size)),
               "dsbt_tdse3d_set_potential")

    def propagate(self, psi: torch.Tensor, F, nsteps: int, hold: int = 1) -> torch.Tensor:
        """In-place propagation by nsteps steps; F: [nsamples][3] field samples (or None)."""
        if psi.dtype != torch.complex128 or not psi.is_cuda or tuple(psi.shape) != (self.nchan, self.N) \
                or not psi.is_contiguous():
            raise ValueError(f"state must be a contiguous complex128 CUDA tensor of shape ({self.nchan}, {self.N})")
        Fp = None if F is None else torch.as_tensor(F).to(device="cuda", dtype=torch.float64).contiguous()
        nb = int(load().dsbt_tdse3d_workspace_size(self._h))
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        _check(load().dsbt_tdse3d_propagate(self._h, _ptr(psi), None if Fp is None else _ptr(Fp), int(nsteps),
                                            int(hold), _ptr(self._ws), self._ws.numel(), _stream()),
               "dsbt_tdse3d_propagate")
        return psi

    def propagate_velocity(self, psi: torch.Tensor, A, nsteps: int, hold: int = 1, F=None) -> torch.Tensor:
        """In-place velocity-gauge propagation; A (and optionally F): [nsamples][3]."""
        if psi.dtype != torch.complex128 or not psi.is_cuda or tuple(psi.shape) != (self.nchan, self.N) \
                or not psi.is_contiguous():
            raise ValueError(f"state must be a contiguous complex128 CUDA tensor of shape ({self.nchan}, {self.N})")
        Ap = torch.as_tensor(A).to(device="cuda", dtype=torch.float64).contiguous()
        Fp = None if F is None else torch.as_tensor(F).to(device="cuda", dtype=torch.float64).contiguous()
        nb = int(load().dsbt_tdse3d_workspace_size(self._h))
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        _check(load().dsbt_tdse3d_propagate_velocity(self._h, _ptr(psi), None if Fp is None else _ptr(Fp), _ptr(Ap),
                                                     int(nsteps), int(hold), _ptr(self._ws), self._ws.numel(),
                                                     _stream()), "dsbt_tdse3d_propagate_velocity")
        return psi

    def gradient(self, psi0: torch.Tensor, F, nsteps: int, hold: int, r_cut: float, K: int = 20):
        """(O, dO/dF): O = sum over r > r_cut of |psi_S|^2 after nsteps length-gauge
        steps from psi0 (unchanged), dO/dF [nsamples][3] by the adjoint method with
        a checkpoint every K steps."""
        if psi0.dtype != torch.complex128 or not psi0.is_cuda or tuple(psi0.shape) != (self.nchan, self.N) \
                or not psi0.is_contiguous():
            raise ValueError(f"state must be a contiguous complex128 CUDA tensor of shape ({self.nchan}, {self.N})")
        Fp = torch.as_tensor(F).to(device="cuda", dtype=torch.float64).contiguous()
        ns = Fp.numel() // 3
        nb = int(load().dsbt_tdse3d_gradient_workspace_size(self._h, int(nsteps), int(K)))
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        O = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty((ns, 3), dtype=torch.float64, device="cuda")
        _check(load().dsbt_tdse3d_gradient(self._h, _ptr(psi0), _ptr(Fp), int(ns), int(nsteps), int(hold),
                                           float(r_cut), int(K), _ptr(O), _ptr(g), _ptr(ws), nb, _stream()),
               "dsbt_tdse3d_gradient")
        return O, g


class Tdse:
    """Split-operator TDSE (m = 0, length gauge) through the DSBT: see
    dsbt_tdse_* in include/dsbt.h.  State: complex128 CUDA tensor [L][N]."""

    def __init__(self, plan: Plan, L: int, tau: float, Z: float = 1.0, a2: float = 0.5, m: int = 0):
        h = ctypes.c_void_p()
        _check(load().dsbt_tdse_create_m(plan.handle, int(L), int(m), float(tau), float(Z), float(a2),
                                         ctypes.byref(h)), "dsbt_tdse_create_m")
        self._h, self.plan, self.L, self.N, self.tau = h, plan, int(L), plan.N, float(tau)
        self._ws = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dsbt_tdse_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_potential(self, V):
        """Radial potential V(r_i) on the plan's midpoint grid (N values)."""
        import numpy as np
        V = np.ascontiguousarray(V, dtype=np.float64)
        _check(load().dsbt_tdse_set_potential(self._h, V.ctypes.data_as(ctypes.c_void_p), int(V.size)),
               "dsbt_tdse_set_potential")

    def angular(self):
        import numpy as np
        eta = np.empty(self.L)
        w = np.empty(self.L)
        P = np.empty((self.L, self.L))
        _check(load().dsbt_tdse_angular(self._h, eta.ctypes.data_as(ctypes.c_void_p),
                                        w.ctypes.data_as(ctypes.c_void_p), P.ctypes.data_as(ctypes.c_void_p)),
               "dsbt_tdse_angular")
        return eta, w, P

    def workspace(self, nsteps: int, K: int = 0) -> torch.Tensor:
        nb = int(load().dsbt_tdse_workspace_size(self._h, int(nsteps), int(K)))
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        return self._ws

    def _state(self, psi):
        if psi.dtype != torch.complex128 or not psi.is_cuda or tuple(psi.shape) != (self.L, self.N) \
                or not psi.is_contiguous():
            raise ValueError(f"state must be a contiguous complex128 CUDA tensor of shape ({self.L}, {self.N})")

    def propagate(self, psi: torch.Tensor, E: torch.Tensor, nsteps: int, hold: int = 1,
                  backward: bool = False) -> torch.Tensor:
        """In-place propagation by nsteps steps (backward=True: the inverse steps)."""
        self._state(psi)
        E = E.to(device="cuda", dtype=torch.float64).contiguous()
        ws = self.workspace(nsteps, 0)
        _check(load().dsbt_tdse_propagate(self._h, _ptr(psi), _ptr(E), int(nsteps), int(hold),
                                          -1.0 if backward else 1.0, _ptr(ws), ws.numel(), _stream()),
               "dsbt_tdse_propagate")
        return psi

    def propagate_velocity(self, psi: torch.Tensor, A: torch.Tensor, nsteps: int, hold: int = 1, E=None,
                           backward: bool = False) -> torch.Tensor:
        """In-place velocity-gauge propagation (dsbt_tdse_propagate_velocity):
        A (and optionally E) per hold steps."""
        self._state(psi)
        A = A.to(device="cuda", dtype=torch.float64).contiguous()
        Ep = None if E is None else E.to(device="cuda", dtype=torch.float64).contiguous()
        ws = self.workspace(nsteps, 0)
        _check(load().dsbt_tdse_propagate_velocity(self._h, _ptr(psi), None if Ep is None else _ptr(Ep), _ptr(A),
                                                   int(nsteps), int(hold), -1.0 if backward else 1.0, _ptr(ws),
                                                   ws.numel(), _stream()), "dsbt_tdse_propagate_velocity")
        return psi

    def observable(self, psi: torch.Tensor, r_cut: float) -> torch.Tensor:
        self._state(psi)
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(load().dsbt_tdse_observable(self._h, _ptr(psi), float(r_cut), _ptr(out), _stream()),
               "dsbt_tdse_observable")
        return out[0]

    def gradient(self, psi0: torch.Tensor, E: torch.Tensor, nsteps: int, hold: int, r_cut: float,
                 K: int = 20):
        """(O, dO/dE) by the checkpointed adjoint (dsbt_tdse_gradient)."""
        self._state(psi0)
        E = E.to(device="cuda", dtype=torch.float64).contiguous()
        O = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(E.numel(), dtype=torch.float64, device="cuda")
        ws = self.workspace(nsteps, K)
        _check(load().dsbt_tdse_gradient(self._h, _ptr(psi0), _ptr(E), int(E.numel()), int(nsteps), int(hold),
                                         float(r_cut), int(K), _ptr(O), _ptr(g), _ptr(ws), ws.numel(),
                                         _stream()), "dsbt_tdse_gradient")
        return O[0], g


class TdseObservable(torch.autograd.Function):
    """O(E) = sum_{r > r_cut} |psi(T)|^2 as a differentiable function of the
    field samples E.  forward: propagate + observable; backward: the adjoint
    run of dsbt_tdse_gradient (checkpoint every K steps)."""

    @staticmethod
    def forward(ctx, E, tdse, psi0, nsteps, hold, r_cut, K):
        psi = psi0.clone()
        tdse.propagate(psi, E, nsteps, hold)
        O = tdse.observable(psi, r_cut).clone()
        ctx.save_for_backward(E)
        ctx.args = (tdse, psi0, nsteps, hold, r_cut, K)
        return O

    @staticmethod
    def backward(ctx, gO):
        (E,) = ctx.saved_tensors
        tdse, psi0, nsteps, hold, r_cut, K = ctx.args
        _, g = tdse.gradient(psi0, E.detach(), nsteps, hold, r_cut, K)
        return gO * g.to(E.dtype), None, None, None, None, None, None
