"""Seeded synthetic inputs for the DSBT workloads.

This module holds no arithmetic of the transform itself: it only samples radial
functions on the midpoint grid r_i = (i - 1/2) dr (Sec. 2.2, Eq. (14)), scaled by
sqrt(dr) as the transform expects (psi_i = psi(r_i) sqrt(dr)), and draws the
random coefficients that define them.  The same arrays are fed to the CUDA path
and to the CPU oracle.

Workloads (shapes and value distributions follow the paper's test functions, the
Gaussian atomic orbitals r^{l+1} exp(-a r^2) of Sec. 3):

* ``orbital``: one real channel per l, psi = r^{l+1} exp(-a r^2), a ~ U[0.5, 2].
* ``gaussian_sum``: complex channels psi = r * sum_{j=1..8} c_j r^l exp(-a_j r^2),
  c_j ~ CN(0, 1), a_j ~ LogU[0.05, 5]; each Gaussian term is normalised before the
  sum and every channel is scaled to unit 2-norm (so FP32 storage never
  overflows for large l).
* ``all_m_counts``: channel counts (2l + 1) * batch for l = 0..l_max.
"""
from __future__ import annotations

import math

import numpy as np

NTERMS = 8


def midpoint_grid(N: int, dr: float) -> np.ndarray:
    """r_i = (i - 1/2) dr, i = 1..N."""
    return (np.arange(1, N + 1, dtype=np.float64) - 0.5) * dr


def all_m_counts(l_max: int, batch: int = 1) -> list:
    """Channels per l when every m = -l..l is present, times a batch factor."""
    return [(2 * l + 1) * batch for l in range(l_max + 1)]


def orbital(seed: int, N: int, r_max: float, ls) -> tuple:
    """Real Gaussian orbitals, one channel per l.  Returns (list of [1][N]
    float64 arrays, list of alphas)."""
    rng = np.random.default_rng(seed)
    dr = r_max / N
    r = midpoint_grid(N, dr)
    out, alphas = [], []
    for l in ls:
        a = float(rng.uniform(0.5, 2.0))
        psi = r ** (l + 1) * np.exp(-a * r * r) * math.sqrt(dr)
        out.append(psi[None, :].copy())
        alphas.append(a)
    return out, alphas


def gaussian_sum_params(seed: int, counts) -> dict:
    """Random coefficients for ``gaussian_sum``: per channel NTERMS complex
    weights c ~ CN(0,1) and exponents a ~ LogU[0.05, 5]."""
    rng = np.random.default_rng(seed)
    total = int(sum(counts))
    c = (rng.standard_normal((total, NTERMS)) + 1j * rng.standard_normal((total, NTERMS))) / math.sqrt(2)
    a = np.exp(rng.uniform(math.log(0.05), math.log(5.0), size=(total, NTERMS)))
    ls = np.repeat(np.arange(len(counts)), counts)
    return {"c": c, "a": a, "l": ls}


def gaussian_sum(seed: int, N: int, dr: float, counts, dtype=np.complex128,
                 device=None, chunk: int = 1024):
    """Complex channels grouped by l (counts[l] channels for each l, l-major).

    With ``device=None`` returns a numpy array [sum(counts)][N]; otherwise a
    torch tensor on that device, evaluated there in float64 in chunks of
    channels and cast to ``dtype`` (a numpy or torch complex dtype)."""
    prm = gaussian_sum_params(seed, counts)
    total = prm["l"].size
    if device is None:
        r = midpoint_grid(N, dr)
        logr = np.log(r)
        out = np.empty((total, N), dtype=np.complex128)
        for s in range(0, total, chunk):
            e = min(total, s + chunk)
            lg = (prm["l"][s:e, None, None] + 1) * logr[None, None, :] \
                - prm["a"][s:e, :, None] * (r * r)[None, None, :]
            lg -= lg.max(axis=2, keepdims=True)
            g = np.exp(lg)
            g /= np.linalg.norm(g, axis=2, keepdims=True)
            z = np.einsum("cj,cjn->cn", prm["c"][s:e], g)
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            out[s:e] = z
        return out.astype(dtype, copy=False)
    import torch
    r = torch.as_tensor(midpoint_grid(N, dr), device=device)
    logr = torch.log(r)
    tdt = dtype if isinstance(dtype, torch.dtype) else {
        np.complex64: torch.complex64, np.complex128: torch.complex128}[np.dtype(dtype).type]
    out = torch.empty((total, N), dtype=tdt, device=device)
    cc = torch.as_tensor(prm["c"], device=device)
    aa = torch.as_tensor(prm["a"], device=device)
    ll = torch.as_tensor(prm["l"], device=device, dtype=torch.float64)
    for s in range(0, total, chunk):
        e = min(total, s + chunk)
        lg = (ll[s:e, None, None] + 1) * logr[None, None, :] - aa[s:e, :, None] * (r * r)[None, None, :]
        lg = lg - lg.amax(dim=2, keepdim=True)
        g = torch.exp(lg)
        g = g / torch.linalg.vector_norm(g, dim=2, keepdim=True)
        z = torch.einsum("cj,cjn->cn", cc[s:e], g.to(torch.complex128))
        z = z / torch.linalg.vector_norm(z, dim=1, keepdim=True)
        out[s:e] = z.to(tdt)
    return out


def random_lines(seed: int, shape, complex_: bool = True) -> np.ndarray:
    """Plain Gaussian random data (no smoothness), for invariance checks."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    if complex_:
        x = x + 1j * rng.standard_normal(shape)
    return x


def tdse_field(seed: int, nsamples: int = 200, amplitude: float = 0.05) -> np.ndarray:
    """Laser-field samples E_j = A sin^2(pi (j + 1/2) / J) u_j, u_j ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    j = np.arange(nsamples)
    return amplitude * np.sin(np.pi * (j + 0.5) / nsamples) ** 2 * rng.uniform(-1.0, 1.0, nsamples)


def grouped_workload(seed: int, ntransforms: int = 64):
    """Uneven batch: per transform N ~ U{512..8192 step 256}, l_max ~ U{8..64}."""
    rng = np.random.default_rng(seed)
    Ns = 256 * rng.integers(2, 33, size=ntransforms)
    lmaxs = rng.integers(8, 65, size=ntransforms)
    return [(int(n), int(l)) for n, l in zip(Ns, lmaxs)]


def sparse_coefficient_values(seed: int, nchan: int, nrows: int) -> np.ndarray:
    """Values [nchan][nrows] ~ CN(0, 1), each channel scaled to unit 2-norm:
    the nonzero entries of coefficient vectors that vanish outside nrows chosen
    storage indices.  Such vectors are inputs of the inverse transform whose
    exact result needs only those rows of T_l (full-size checks)."""
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal((nchan, nrows)) + 1j * rng.standard_normal((nchan, nrows))) / math.sqrt(2)
    return v / np.linalg.norm(v, axis=1, keepdims=True)
