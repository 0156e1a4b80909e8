#!/usr/bin/env python
"""Throughput benchmark of the GB300 DSBT.

Workload (the precision form): N = 4096 points, r_max = 409.6 (dr = 0.1),
l = 0..63 with all m, batch 8 -> 32768 complex64 channels of seeded Gaussian-sum
radial functions.  One step = one pass of the hot path over the whole batch:
the kinetic round trip F_l -> T_l (with exp(-i k^2 tau/2) in its epilogue) ->
T_l^T -> F_l^T (dsbt_kinetic_grouped), i.e. two channel-transforms per channel.

Printed JSON line (rank 0):
  value       channel-transforms/s of the split-TF32 path, inputs resident in HBM
  e2e         same metric through the public API with pinned HOST buffers
              (dsbt_kinetic_grouped_host: copies inside the call, overlapped in chunks)
              (host->device copy of the inputs and device->host copy of the
              result inside the timed region)
  roofline    of the dominant kernel (the split contraction through the
              interval scheme of DSBT_PLAN_FAST_TF32; --dense: the dense one),
              timed live with CUDA events on its launch stream during the
              timed steps; HBM-bound, algorithmic bytes 16 N B per complex64
              channel-transform (its share per launch), with the whole-step
              fraction and the kernel's tensor rate (algorithmic flops of the
              scheme it runs) against the measured matmul rate beside it
  measured_peaks  FP64 / TF32 / FP16 matmul rates and pinned copy bandwidth
              measured in this run (the denominators MEASURED_PEAKS.json lacks)
  dense_tf32  the same step with the dense split-TF32 contraction
  fp64_gpu    the plain FP64 GPU path on a one-eighth sample (batch 1), and the
              split-TF32 error against it (max |diff| / ||psi|| per channel)
  cpu_baseline  the FP64 CPU oracle on a bounded sample (N = 4096, l = 1, 2),
              one channel per call over all host cores

--impl reference runs the FP64 CPU oracle (the only reference this project
has) on the same workload, a bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DSBT channel-transforms/s vs plain FP64 GPU at ≤1e-6 rel err; % roofline"
UNIT = "channel-transforms/s"
WORKLOADS = {
    # the bench workload (one GPU)
    "precision": dict(N=4096, R_MAX=409.6, L_MAX=63, BATCH=8,
                      desc="precision form: N=4096, r_max=409.6, l=0..63 all m x batch 8 = 32768 complex64 "
                           "Gaussian-sum channels; step = kinetic round trip F, T (+exp(-i k^2 tau/2)), T^T, F^T"),
    # a smaller case of the same kernels for profiler captures (inputs still > L2)
    "small": dict(N=2048, R_MAX=204.8, L_MAX=31, BATCH=8,
                  desc="profiling case: N=2048, r_max=204.8, l=0..31 all m x batch 8 = 8192 complex64 channels"),
    # non-power-of-two grids (radix-Q sine/cosine stages) for profiler captures, inputs > L2
    "grid7936": dict(N=7936, R_MAX=793.6, L_MAX=1, BATCH=800,
                     desc="profiling case: N=7936 (256 x 31), l=0..1 all m x batch 800 = 3200 complex64 channels"),
    "grid4352": dict(N=4352, R_MAX=435.2, L_MAX=1, BATCH=1500,
                     desc="profiling case: N=4352 (256 x 17), l=0..1 all m x batch 1500 = 6000 complex64 channels"),
}
TAU = 0.05
N, R_MAX, L_MAX, BATCH = 4096, 409.6, 63, 8
DR = R_MAX / N
WORKLOAD = WORKLOADS["precision"]["desc"]
FLOP_PER_CHANNEL = 6.0 * N * N   # split-TF32 contraction, one direction, per complex channel


def select_workload(name):
    global N, R_MAX, L_MAX, BATCH, DR, WORKLOAD, FLOP_PER_CHANNEL
    w = WORKLOADS[name]
    N, R_MAX, L_MAX, BATCH = w["N"], w["R_MAX"], w["L_MAX"], w["BATCH"]
    DR = R_MAX / N
    WORKLOAD = w["desc"]
    FLOP_PER_CHANNEL = 6.0 * N * N


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def source_hash(paths):
    m = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:16]


def fast_tf32_mac_per_line(N, l, leaf=128):
    """Multiply-adds of one DSBT_PLAN_FAST_TF32 contraction of one real line of
    T_l as the scheme runs it: near-field triangle of each 128-row leaf, far
    field (l per set bit of the leaf index), moments of the used intervals
    (l per point of half the columns at each level) and of the right intervals
    (l per column right of leaf 0), and the completion rows n < n0_l =
    (l + 2) // 2 (leaf 0's columns plus l per right interval)."""
    nleaf = N // leaf
    levels = (nleaf - 1).bit_length()
    ne = (l + 2) // 2 - (1 if l % 2 == 0 else 0)
    near = sum(r % leaf + 1 for r in range(ne, N))
    far = sum(l * bin(r // leaf).count("1") for r in range(ne, N))
    moments = levels * (N // 2) * l + ((N - leaf) * l if ne else 0)
    completion = ne * (leaf + levels * l)
    return near + far + moments + completion


def ncu_traffic(name="contract_tf32x3_precision_form.json"):
    """DRAM bytes per launch of the contraction from the committed ncu summary,
    if it was taken on the current kernel sources (else None)."""
    prof = os.path.join(ROOT, "profiles", name)
    try:
        with open(prof) as fh:
            d = json.load(fh)
        if d.get("source_sha256_16") != source_hash(d["source_files"]):
            return None
        return d.get("dram_bytes_per_launch_full_size")
    except Exception:
        return None


def probe_peaks(torch, dev):
    """Measured denominators that MEASURED_PEAKS.json lacks, on this GPU:
    dense FP64, TF32 and FP16 matmul rates (torch.matmul, 8192^3, 2 N^3 flop,
    best of several, CUDA events; burst figures) and the pinned host<->device
    copy bandwidth (1 GiB, best of 5)."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def best_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {}
    n = 8192
    old_tf32 = torch.backends.cuda.matmul.allow_tf32
    for name, dt, reps, tf32 in (("fp64", torch.float64, 3, False), ("tf32", torch.float32, 10, True),
                                 ("fp16", torch.float16, 10, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=torch.float32).to(dt)
        b = torch.randn(n, n, device=dev, dtype=torch.float32).to(dt)
        c = torch.empty(n, n, device=dev, dtype=dt)
        ms = best_ms(lambda: torch.matmul(a, b, out=c), reps)
        out[f"{name}_tflops"] = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = old_tf32
    nb = 1 << 30
    h = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d = torch.empty(nb, dtype=torch.uint8, device=dev)
    out["h2d_gbs"] = nb / (best_ms(lambda: d.copy_(h, non_blocking=True), 5) * 1e-3) / 1e9
    out["d2h_gbs"] = nb / (best_ms(lambda: h.copy_(d, non_blocking=True), 5) * 1e-3) / 1e9
    # both directions at once (another pinned pair, a second stream): the bound of
    # a step that copies its inputs in and its results out concurrently
    h2 = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d2 = torch.empty(nb, dtype=torch.uint8, device=dev)
    s2 = torch.cuda.Stream()

    def both():
        s2.wait_stream(st)
        d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        st.wait_stream(s2)
    out["bidir_gbs_each_way"] = nb / (best_ms(both, 5) * 1e-3) / 1e9
    del h, d, h2, d2
    torch.cuda.empty_cache()
    out["how"] = ("torch.matmul 8192^3 (2 N^3 flop), best of 3 (fp64) / 10 (tf32 with allow_tf32, fp16), "
                  "CUDA events; pinned 1 GiB copies best of 5, one way and both ways at once")
    return out


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            self.file.seek(0)
            for line in self.file.read().splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            self.file.close()
            os.unlink(self.file.name)
        return rows

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if s is not None]
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def bad_clocks(c):
    if any(r in c.get("reasons", []) for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")):
        return True
    if c.get("sm_mhz") and c.get("sm_max_mhz") and c["sm_mhz"] < 0.5 * c["sm_max_mhz"] and not c["reasons"]:
        return True
    return False


# ---------------------------------------------------------------- CPU oracle leg

def oracle_threads():
    return max(1, os.cpu_count() or 1)


def oracle_sample(per_thread=2, ls=(1, 2), seed=11):
    """Times the FP64 oracle as it stands on a bounded sample, one channel per
    call of its C routines spread over all host cores by a thread pool (the C
    routines release the GIL; the oracle's arithmetic is untouched): for each l
    in ls, per_thread x cores channels of the workload's Gaussian-sum inputs,
    kinetic round trip by naive O(N^2) sums.  The cost per channel does not
    depend on l (dense sums), so the sample stands for every l group; the
    factor build (binary128 DLOP rows, explicit F_l), which does depend on l,
    is timed separately and excluded.  Returns (transforms, seconds, build_s,
    threads)."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    from paper_1509_07115_gb300 import inputs
    nt = oracle_threads()
    nchan = per_thread * nt
    counts = [0] * (max(ls) + 1)
    for l in ls:
        counts[l] = nchan
    x = inputs.gaussian_sum(seed, N, DR, counts)
    t0 = time.perf_counter()
    FT = {l: (oracle.F_matrix(N, l), oracle.T_matrix(N, l)) for l in ls}
    t_build = time.perf_counter() - t0
    jobs = []
    c0 = 0
    for l in range(max(ls) + 1):
        for c in range(counts[l]):
            jobs.append((l, c0 + c))
        c0 += counts[l]

    def one(job):
        l, c = job
        F, T = FT[l]
        kt = oracle.k_tilde(N, R_MAX, l)
        b = oracle.apply(T, oracle.apply(F, x[c:c + 1])) * np.exp(-0.5j * kt * kt * TAU)
        oracle.apply(F, oracle.apply(T, b, transpose=True), transpose=True)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(nt) as ex:
        list(ex.map(one, jobs))
    t_xform = time.perf_counter() - t0
    return 2 * len(jobs), t_xform, t_build, nt


def gpu_local_cpus(index: int):
    """CPU cores local to GPU `index` (the "CPU Affinity" column of
    `nvidia-smi topo -m`), or None.  Pinned host buffers are first touched by
    the allocating thread, so running the host side there keeps the pinned
    memory of the host-streamed leg on the GPU's own NUMA node."""
    try:
        txt = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=20).stdout
    except Exception:
        return None
    lines = [ln for ln in txt.splitlines() if ln.strip()]
    hdr = next((ln for ln in lines if "CPU Affinity" in ln), None)
    if hdr is None:
        return None
    cols = [c.strip() for c in hdr.split("\t")]
    row = next((ln for ln in lines if ln.split("\t")[0].strip() == f"GPU{index}"), None)
    if row is None:
        return None
    cells = [c.strip() for c in row.split("\t")]
    try:
        spec = cells[cols.index("CPU Affinity")]
    except (ValueError, IndexError):
        return None
    cpus = set()
    try:
        for part in spec.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    except ValueError:
        return None
    return sorted(cpus & set(os.sched_getaffinity(0))) or None


def rank_seed(rank: int, base: int = 100) -> int:
    """Seed of a rank's synthetic batch: every rank transforms its own batch of
    the workload (weak scaling, no data-path collective)."""
    return base + rank


def job_ms(ms_local: float, world: int, dist, device) -> float:
    """Duration of the timed region for the whole job: the max over ranks."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step: float, world: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return units_per_rank_step * world * steps / (ms_max * 1e-3)


def run_reference(args, rank):
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    import numpy as np
    from paper_1509_07115_gb300 import inputs
    # factors for the sampled l, built once (binary128 recurrences); each step
    # then runs the kinetic round trip of one channel per host core (threads,
    # alternating l = 1 and 2); the dense sums cost the same for every l
    nt = oracle_threads()
    t0 = time.perf_counter()
    FT = {1: (oracle.F_matrix(N, 1), oracle.T_matrix(N, 1)), 2: (oracle.F_matrix(N, 2), oracle.T_matrix(N, 2))}
    t_build = time.perf_counter() - t0
    x = inputs.gaussian_sum(13, N, DR, [0, nt, nt])

    def one(c):
        l = 1 + (c % 2)
        F, T = FT[l]
        xs = x[(l - 1) * nt + c // 2:(l - 1) * nt + c // 2 + 1]
        kt = oracle.k_tilde(N, R_MAX, l)
        b = oracle.apply(T, oracle.apply(F, xs)) * np.exp(-0.5j * kt * kt * TAU)
        oracle.apply(F, oracle.apply(T, b, transpose=True), transpose=True)

    ex = ThreadPoolExecutor(nt)

    def step():
        list(ex.map(one, range(nt)))
        return 2 * nt
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    ntr = 0
    for _ in range(args.steps):
        ntr += step()
    dt = time.perf_counter() - t0
    ex.shutdown()
    value = ntr / dt
    sample = (f"{nt} complex channels per step (one per host thread, alternating l=1 and l=2) of the N=4096 "
              f"workload, kinetic round trip by naive O(N^2) sums (cost independent of l); factor build for "
              f"l=1,2 took {t_build:.1f} s (excluded)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian-sum radial functions)",
            "config": {"workload": WORKLOAD, "N": N, "l_max": L_MAX, "channels": sum(2 * l + 1 for l in range(L_MAX + 1)) * BATCH,
                       "reference": "FP64 CPU oracle (plain C, binary128 DLOP rows), bounded sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- TDSE leg



def fast64_fma_per_line(N, l, B=64):
    """Useful multiply-adds of one FAST64 contraction of one real line of T_l
    (forward and inverse cost the same): near-field triangle of each leaf,
    far field (l per set bit of the leaf index), direct moments of the used
    intervals (l per point of half the columns at each level), and the dense
    completion rows n < n0_l = (l + 2) // 2."""
    nleaf = N // B
    levels = (nleaf - 1).bit_length()
    ne = (l + 2) // 2 - (1 if l % 2 == 0 else 0)
    near = sum(r % B + 1 for r in range(ne, N))
    far = sum(l * bin(r // B).count("1") for r in range(ne, N))
    return near + far + levels * (N // 2) * l + ne * N


def tdse_leg(dsbt, inputs, torch, dev, fp64_peak):
    """m = 0, l = 0..63, N = 2048, dr = 0.1, soft-Coulomb, 400 steps of 0.05 with
    200 field samples (held 2 steps): propagation and adjoint-gradient timings,
    and the FP64 contraction's rate against the measured FP64 matmul rate."""
    import numpy as np
    Nt, L, tau, steps = 2048, 64, 0.05, 400
    plan = dsbt.Plan(Nt, 204.8, L - 1, tf32x3=False)
    td = dsbt.Tdse(plan, L, tau)
    c0 = np.zeros((L, Nt), dtype=np.complex128)
    r = (np.arange(Nt) + 0.5) * 0.1
    f = r * np.exp(-0.5 * r * r) * np.sqrt(0.1)
    c0[0] = f / np.linalg.norm(f)
    psi0 = torch.from_numpy(c0).to(dev)
    E = torch.from_numpy(inputs.tdse_field(7, 200)).to(dev)
    psi = psi0.clone()
    td.propagate(psi, E, 20, 2)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    psi = psi0.clone()
    dsbt.profile_enable(True)
    e0.record(st)
    td.propagate(psi, E, steps, 2)
    e1.record(st)
    torch.cuda.synchronize()
    prop_ms = e0.elapsed_time(e1)
    prof = dsbt.profile_read()
    dsbt.profile_enable(False)
    drift = abs(torch.linalg.vector_norm(psi).item() - 1.0)
    e0.record(st)
    O, g = td.gradient(psi0, E, steps, 2, 50.0, K=20)
    e1.record(st)
    torch.cuda.synchronize()
    grad_ms = e0.elapsed_time(e1)
    n64, ms64 = prof.get("contract_f64", (1, 0.0))
    flop = 2.0 * 2 * L * Nt * Nt / 2   # per launch: 2 real lines x N^2/2 MACs x 2 flop, 64 channels
    achieved = flop / (ms64 / n64 * 1e-3) / 1e12
    td.close()
    plan.close()
    # the same propagation with the O(N l log N) FP64 contraction (DSBT_PLAN_FAST64)
    fplan = dsbt.Plan(Nt, 204.8, L - 1, tf32x3=False, fast64=True)
    ftd = dsbt.Tdse(fplan, L, tau)
    psif = psi0.clone()
    ftd.propagate(psif, E, 20, 2)
    torch.cuda.synchronize()
    psif = psi0.clone()
    dsbt.profile_enable(True)
    e0.record(st)
    ftd.propagate(psif, E, steps, 2)
    e1.record(st)
    torch.cuda.synchronize()
    fast_ms = e0.elapsed_time(e1)
    fprof = dsbt.profile_read()
    dsbt.profile_enable(False)
    fast_dev = (psif - psi).abs().max().item()
    fast_flop = 2 * 2 * 2 * sum(fast64_fma_per_line(Nt, l) for l in range(L))   # 2 lines, fwd + inv
    fast_achieved = fast_flop / (fprof["contract_f64"][1] / steps * 1e-3) / 1e12
    ftd.close()
    fplan.close()
    # all m (Y = P Phi): 32 x 17 = 544 channels, field along x
    p3 = dsbt.Plan(Nt, 204.8, 40, tf32x3=False, fast64=True)
    t3 = dsbt.Tdse3d(p3, 32, 8, tau)
    r3 = (np.arange(Nt) + 0.5) * 0.1
    t3.set_potential(-1.0 / np.sqrt(r3 * r3 + 0.5))
    c3 = np.zeros((t3.nchan, Nt), dtype=np.complex128)
    c3[t3.channels.index((0, 0))] = f / np.linalg.norm(f)
    F3 = torch.zeros((200, 3), dtype=torch.float64, device=dev)
    F3[:, 0] = E[:200]
    psi3 = torch.from_numpy(c3).to(dev)
    t3.propagate(psi3, F3, 10, 2)
    torch.cuda.synchronize()
    steps3 = 100
    dsbt.profile_enable(True)
    e0.record(st)
    t3.propagate(psi3, F3, steps3, 2)
    e1.record(st)
    torch.cuda.synchronize()
    ms3 = e0.elapsed_time(e1)
    prof3 = dsbt.profile_read()
    dsbt.profile_enable(False)
    norm3 = torch.linalg.vector_norm(psi3).item()
    # adjoint gradient of the norm beyond r = 50 over the 3 x 50 field components
    psi30 = torch.from_numpy(c3).to(dev)
    e0.record(st)
    O3, g3 = t3.gradient(psi30, F3[:50], steps3, 2, 50.0, K=10)
    e1.record(st)
    torch.cuda.synchronize()
    grad3_ms = e0.elapsed_time(e1)
    t3.close()
    p3.close()
    return {"config": "m=0, l=0..63, N=2048, dr=0.1, 400 steps of 0.05, soft-Coulomb -1/sqrt(r^2+0.5), "
                      "200 field samples held 2 steps, observable = norm beyond r=50, checkpoint every 20",
            "propagate_ms_per_step": prop_ms / steps, "gradient_ms_total": grad_ms,
            "norm_drift_400_steps": drift, "observable": O.item(),
            "kernels_ms_per_step": {k: v[1] / steps for k, v in prof.items()},
            "all_m": {"config": "N=2048, L=32 per m, M=8 (544 channels, l <= 39), field along x, "
                                "100 steps of 0.05, DSBT_PLAN_FAST64 plan", "propagate_ms_per_step": ms3 / steps3,
                      "kernels_ms_per_step": {k: v[1] / steps3 for k, v in prof3.items()},
                      "norm_after": norm3,
                      "gradient_ms_total": grad3_ms, "gradient_observable": O3.item(),
                      "gradient_config": "dO/dF over 50 samples x 3 components, O = norm beyond r = 50, "
                                         "checkpoint every 10 steps"},
            "fast64": {"propagate_ms_per_step": fast_ms / steps,
                       "kernels_ms_per_step": {k: v[1] / steps for k, v in fprof.items()},
                       "max_abs_diff_vs_dense": fast_dev,
                       "roofline_contract": {"bound": "fp64", "achieved": fast_achieved,
                                             "peak": fp64_peak, "unit": "TFLOP/s",
                                             "frac": fast_achieved / fp64_peak,
                                             "flop_per_step": fast_flop,
                                             "peak_source": "measured fp64 matmul (burst, this run)"}},
            "roofline_contract_f64": {"bound": "fp64", "achieved": achieved, "peak": fp64_peak,
                                      "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                                      "peak_source": "measured fp64 matmul (burst, this run)"}}


# ---------------------------------------------------------------- plain FP64 leg (C2)

def c2_leg(dsbt, inputs, torch, dev, steps=5):
    """Plain FP64 complex128 DSBT: N = 2048, r_max = 204.8, l <= 31 all m (1024
    channels, seeded Gaussian sums), forward + inverse round trip per step, on
    the O(N l log N) FP64 plan (DSBT_PLAN_FAST64) and on the dense FP64 plan."""
    N2, R2, L2 = 2048, 204.8, 31
    counts = inputs.all_m_counts(L2, 1)
    n = sum(counts)
    x = inputs.gaussian_sum(400, N2, R2 / N2, counts, dtype=torch.complex128, device=dev)
    nrm = torch.linalg.vector_norm(x, dim=1)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"config": "N=2048, r_max=204.8, l=0..31 all m = 1024 complex128 channels; step = forward + inverse",
           "unit": UNIT}
    for name, fast in (("fast64", True), ("dense_fp64", False)):
        p = dsbt.Plan(N2, R2, L2, fp64=True, tf32x3=False, fast64=fast)
        ws = torch.empty(p.workspace_bytes(n, torch.complex128), dtype=torch.uint8, device=dev)
        b = torch.empty_like(x)
        y = torch.empty_like(x)
        for _ in range(2):
            p.forward_grouped(counts, x, out=b, workspace=ws)
            p.inverse_grouped(counts, b, out=y, workspace=ws)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            p.forward_grouped(counts, x, out=b, workspace=ws)
            p.inverse_grouped(counts, b, out=y, workspace=ws)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        err = ((y - x).abs().amax(dim=1) / nrm).max().item()
        res[name] = {"value": 2 * n / (ms * 1e-3), "ms_per_step": ms, "round_trip_max_rel_err": err}
        p.close()
        del ws, b, y
    return res


# ---------------------------------------------------------------- uneven batch leg

def batch_leg(dsbt, inputs, torch, dev, steps, warmup, peak, scheme="interval"):
    """64 transforms, N ~ U{512..8192 step 256}, l_max ~ U{8..64} (seed 0), 2l+1
    complex64 Gaussian-sum channels per l; one kinetic step of the whole batch
    per graph replay.  scheme "dense": factors shared across grids, one
    persistent contraction launch per direction, tile order and width
    autotuned; "interval": one interval-scheme plan per distinct grid, the
    transforms' grouped calls forked over internal streams inside the graph."""
    work = inputs.grouped_workload(0)
    trs = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in work]
    dr = 0.1
    t0 = time.perf_counter()
    b = dsbt.Batch(trs, dr, autotune=True, scheme=scheme)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    xs = [inputs.gaussian_sum(300 + k, N, dr, c, dtype=torch.complex64, device=dev).reshape(-1)
          for k, (N, lm, c) in enumerate(trs)]
    x = torch.cat(xs)
    del xs
    y = torch.empty_like(x)
    g = b.capture_kinetic(x, TAU, y)
    for _ in range(warmup):
        b.launch_graph(g)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dsbt.profile_enable(True)
    # launches inside a graph are not traced; time one direct call for the kernel split
    b.kinetic(x, TAU, out=y)
    torch.cuda.synchronize()
    prof = dsbt.profile_read()
    dsbt.profile_enable(False)
    e0.record(st)
    for _ in range(steps):
        b.launch_graph(g)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nchan = sum(sum(c) for _, _, c in trs)
    flop = sum(6.0 * N * N * sum(c) for N, _, c in trs)   # dense count, per contraction launch (one direction)
    n_c, ms_c = prof.get("contract_tf32x3", (1, 0.0))
    info = b.info()
    # sampled parity: one mid-size transform against the single-plan path
    k = max(range(len(trs)), key=lambda i: (trs[i][0] <= 2048, trs[i][0]))
    N, lm, c = trs[k]
    p = dsbt.Plan(N, N * dr, lm, fp64=False)
    off = b.offsets()[k]
    xk = x[off:off + sum(c) * N].reshape(-1, N)
    ref = p.kinetic_grouped(c, xk, TAU)
    yk = y[off:off + sum(c) * N].reshape(-1, N)
    err = ((yk - ref).abs().amax(dim=1) / torch.linalg.vector_norm(xk, dim=1)).max().item()
    p.close()
    b.close()
    del x, y
    torch.cuda.empty_cache()
    bytes_step = 2 * 16.0 * sum(N * sum(c) for N, _, c in trs)
    out = {"scheme": scheme,
           "config": "64 transforms, N ~ U{512..8192 step 256}, l_max ~ U{8..64} (seed 0), 2l+1 complex64 "
                     "Gaussian-sum channels per l, dr = 0.1; one graph replay = kinetic step of the batch",
           "channels": nchan, "value": 2 * nchan / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": steps, "build_s": build_s,
           "kernels_ms_direct_call": {kk: v[1] for kk, v in prof.items()},
           "hbm": {"algorithmic_bytes_per_step": bytes_step,
                   "frac_whole_step": bytes_step / (ms * 1e-3) / 1e9 / load_peaks()[0]["hbm_gbs"]},
           "max_rel_err_vs_single_plan": err}
    if scheme == "dense":
        ach = flop / (ms_c / n_c * 1e-3) / 1e12
        out["autotune"] = info
        out["roofline_contract"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                    "frac": ach / peak, "flop_per_launch": flop,
                                    "note": "dense N^2 flops of the contraction this batch runs",
                                    "peak_source": "measured tf32 matmul (burst, this run)"}
    else:
        out["note"] = ("kernel times of the direct call are summed over the internal streams, which overlap")
    return out


# ---------------------------------------------------------------- GPU leg

def dense_leg(dsbt, torch, counts, x, peak, args):
    """The same kinetic step with the dense split-TF32 contraction (a plan
    without DSBT_PLAN_FAST_TF32), for comparison with the interval scheme."""
    nchan = sum(counts)
    p = dsbt.Plan(N, R_MAX, L_MAX, fp64=False, tf32x3=True)
    y = torch.empty_like(x)
    ws = p.workspace(nchan, torch.complex64)
    for _ in range(3):
        p.kinetic_grouped(counts, x, TAU, out=y, workspace=ws)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 3)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dsbt.profile_enable(True)
    e0.record(st)
    for _ in range(steps):
        p.kinetic_grouped(counts, x, TAU, out=y, workspace=ws)
    e1.record(st)
    torch.cuda.synchronize()
    prof = dsbt.profile_read()
    dsbt.profile_enable(False)
    ms = e0.elapsed_time(e1) / steps
    n_c, ms_c = prof.get("contract_tf32x3", (0, 0.0))
    ach = FLOP_PER_CHANNEL * nchan / (ms_c / max(1, n_c) * 1e-3) / 1e12
    p.close()
    del ws
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": 2 * nchan / (ms * 1e-3), "unit": UNIT,
            "contraction_ms_per_step": ms_c / steps,
            "roofline": {"bound": "tensor", "kernel": "contract_tf32x3", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach / peak, "flop_per_launch": FLOP_PER_CHANNEL * nchan}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tdse", action="store_true", help="skip the TDSE propagation/adjoint leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch leg")
    ap.add_argument("--e2e-chunks", type=int, default=16, help="chunks of the host-streamed e2e call")
    ap.add_argument("--fast-lag", type=int, default=0,
                    help="tile order of the interval-scheme contraction (dsbt_plan_set_fast_lag; 0: the default)")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the matmul / copy probes (profiler runs); fractions then use nominal ratios")
    ap.add_argument("--dense", action="store_true",
                    help="time the dense split-TF32 contraction instead of the interval scheme")
    ap.add_argument("--workload", default="precision", choices=sorted(WORKLOADS),
                    help="'small' is a reduced case for profiler captures, not a bench line")
    args = ap.parse_args()
    select_workload(args.workload)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    from paper_1509_07115_gb300 import dsbt, inputs

    cpus = gpu_local_cpus(local)
    if cpus:
        os.sched_setaffinity(0, cpus)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    counts = inputs.all_m_counts(L_MAX, BATCH)
    nchan = sum(counts)

    def barrier():
        if world > 1:
            dist.barrier()

    fast = not args.dense
    # FP64 factors with the O(N l log N) FP64 scheme for the FP64 comparison leg
    # (needs N / 64 a power of two)
    fast64 = (not args.no_fp64) and (N // 64) & (N // 64 - 1) == 0 and N % 64 == 0
    plan = dsbt.Plan(N, R_MAX, L_MAX, fp64=not args.no_fp64, tf32x3=not fast, fast_split=fast, fast64=fast64)
    if fast and args.fast_lag > 0:
        plan.set_fast_lag(args.fast_lag)
    x = inputs.gaussian_sum(rank_seed(rank), N, DR, counts, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    ws = plan.workspace(nchan, torch.complex64)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.kinetic_grouped(counts, x, TAU, out=y, workspace=ws)
    torch.cuda.synchronize()

    def timed_region():
        dsbt.profile_enable(True)
        n0 = dsbt.launch_count()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.kinetic_grouped(counts, x, TAU, out=y, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = dsbt.launch_count() - n0
        prof = dsbt.profile_read()
        dsbt.profile_enable(False)
        return e0.elapsed_time(e1), launches, prof

    sampler = ClockSampler(local)
    sampler.start()
    ms, launches, prof = timed_region()
    clocks = ClockSampler.summarize(sampler.stop())
    if bad_clocks(clocks):
        sampler = ClockSampler(local)
        sampler.start()
        ms, launches, prof = timed_region()
        clocks = ClockSampler.summarize(sampler.stop())
        clocks["remeasured"] = True
    status = plan.device_status()
    if status != 0:
        raise RuntimeError(f"device status {status} after the timed region")

    ms_max = job_ms(ms, world, dist, dev)
    value = job_value(2 * nchan, world, args.steps, ms_max)

    # ---------------------------------------------------------- e2e via host buffers
    # dsbt_kinetic_grouped_host: pinned host input and output, the library streams
    # the channels through the GPU in chunks (copies overlap the transforms)
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    hws = plan.host_workspace(counts, torch.complex64, chunks=args.e2e_chunks)
    for _ in range(2):
        plan.kinetic_grouped_host(counts, xh, TAU, out=yh, chunks=args.e2e_chunks, workspace=hws)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # about a second of calls: the host link stalls for 20-30 ms roughly every 0.5 s (with any
    # chunk count), so a short window reads either above or below the long-run mean
    e2e_steps = max(3, 5 * args.steps)
    e0.record(stream)
    for _ in range(e2e_steps):
        plan.kinetic_grouped_host(counts, xh, TAU, out=yh, chunks=args.e2e_chunks, workspace=hws)
    e1.record(stream)
    torch.cuda.synchronize()
    job_ms_e2e = job_ms(e0.elapsed_time(e1), world, dist, dev)
    e2e_value = job_value(2 * nchan, world, e2e_steps, job_ms_e2e)
    nbytes = x.numel() * x.element_size()
    del hws

    # ---------------------------------------------------------- measured peaks (after the timed region)
    peaks, src = load_peaks()
    if args.no_probe:   # nominal ratios to the measured BF16 rate; no copy figures
        bf = peaks["bf16_tflops"]
        probes = {"fp64_tflops": bf * 1.25 / 2250, "tf32_tflops": bf * 1.1 / 2.25, "fp16_tflops": bf,
                  "h2d_gbs": None, "d2h_gbs": None, "bidir_gbs_each_way": None,
                  "how": "not probed: nominal ratios to bf16_tflops"}
    else:
        probes = probe_peaks(torch, dev)
    hbm = peaks["hbm_gbs"]

    # ---------------------------------------------------------- roofline of the contraction
    # The method's algorithmic work is HBM-bound: 16 N bytes per complex64
    # channel-transform (one read and one write of the channel), i.e.
    # 2 x 16 N x channels bytes per kinetic step.  A launch of the dominant
    # kernel is credited with its share of the step's bytes (step bytes over the
    # contraction launches per step); its tensor rate against the measured dense
    # rate of its operand type is reported beside it.
    k_launches, k_ms = prof.get("contract_tf32x3", (0, 0.0))
    avg_ms = k_ms / max(1, k_launches)
    launches_per_step = k_launches / args.steps
    bytes_step = 2 * 16.0 * N * nchan
    bytes_launch = bytes_step / launches_per_step
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    if fast:
        # two launches per step (forward: moments and rows; adjoint: weights and
        # columns, each pair interleaved in one launch); algorithmic flops of the
        # interval scheme, 3 split products
        flop_per_step = 2 * 3 * 2.0 * sum(2 * c * fast_tf32_mac_per_line(N, l) for l, c in enumerate(counts))
        kname, tname = "contract_ftc (interval scheme, DSBT_PLAN_FAST_SPLIT)", "contract_ftc_precision_form.json"
    else:
        flop_per_step = 2 * FLOP_PER_CHANNEL * nchan
        kname, tname = "contract_tf32x3", "contract_tf32x3_precision_form.json"
    flop_per_launch = flop_per_step / launches_per_step
    tflops = flop_per_launch / (avg_ms * 1e-3) / 1e12
    # the interval scheme multiplies FP16 pairs, the dense kernel TF32 pairs
    tpeak = probes["fp16_tflops"] if fast else probes["tf32_tflops"]
    tpeak_src = "measured fp16 matmul (burst, this run)" if fast else "measured tf32 matmul (burst, this run)"
    traffic = ncu_traffic(tname) if args.workload == "precision" else None
    step_ms = ms / args.steps
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
                "algorithmic_bytes_per_launch": bytes_launch,
                "algorithmic_bytes_rule": "16 N B per complex64 channel-transform, 2 per channel per step, "
                                          "shared over the contraction launches of the step",
                "traffic_ratio": (traffic / bytes_launch) if traffic else None,
                # the rate at which the launch moves its measured DRAM bytes
                "traffic_gbs": (traffic / (avg_ms * 1e-3) / 1e9) if traffic else None,
                "traffic_frac": (traffic / (avg_ms * 1e-3) / 1e9 / hbm) if traffic else None,
                "avg_launch_ms": avg_ms, "launches_per_step": launches_per_step,
                "whole_step": {"achieved": bytes_step / (step_ms * 1e-3) / 1e9, "frac": bytes_step / (step_ms * 1e-3) / 1e9 / hbm,
                               "ms": step_ms},
                "tensor": {"achieved": tflops, "peak": tpeak, "unit": "TFLOP/s", "frac": tflops / tpeak,
                           "flop_per_launch": flop_per_launch,
                           "peak_source": tpeak_src,
                           "dense_equivalent_tflops": 2 * FLOP_PER_CHANNEL * nchan / (k_ms / args.steps * 1e-3) / 1e12},
                "kernels_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()}}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (split-fp16 interval-scheme contraction, fp32 accumulate)" if fast else "f32 (split-tf32 contraction, fp32 accumulate)",
                "data": "synthetic (seeded Gaussian-sum radial functions r sum_j c_j r^l exp(-a_j r^2))",
                "config": {"workload": WORKLOAD, "N": N, "r_max": R_MAX, "l_max": L_MAX, "batch": BATCH,
                           "channels_per_gpu": nchan, "tau": TAU,
                           "l2": "inputs larger than L2 (1.07 GB in + 1.07 GB out per step per GPU)",
                           "host_cpus": f"{cpus[0]}-{cpus[-1]} ({len(cpus)} cores local to the GPU)" if cpus
                           else "not pinned"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                        "api": f"dsbt_kinetic_grouped_host, pinned host buffers, {args.e2e_chunks} chunks"},
                "gpu_launches": launches, "roofline": roofline, "clocks": clocks,
                "measured_peaks": dict(probes, hbm_gbs=hbm, bf16_tflops=peaks.get("bf16_tflops"),
                                       bf16_tflops_sustained=peaks.get("bf16_tflops_sustained"))}
        if probes["h2d_gbs"]:
            line["e2e"]["copy_bound"] = {
                "h2d_gbs_achieved": nbytes / (1e-3 * job_ms_e2e / e2e_steps) / 1e9,
                "h2d_gbs_pinned_peak": probes["h2d_gbs"], "d2h_gbs_pinned_peak": probes["d2h_gbs"],
                "bidir_gbs_each_way_peak": probes["bidir_gbs_each_way"],
                "note": "each step copies the batch in and out; copies run both ways at once, overlapped with compute"}

    # ---------------------------------------------------------- FP64 GPU path (sample) + error
    if not args.no_fp64:
        counts1 = inputs.all_m_counts(L_MAX, 1)
        n1 = sum(counts1)
        x64 = inputs.gaussian_sum(200 + rank, N, DR, counts1, dtype=torch.complex128, device=dev)
        y64 = torch.empty_like(x64)

        def time_fp64(p):
            ws64 = torch.empty(p.workspace_bytes(n1, torch.complex128), dtype=torch.uint8, device=dev)
            p.kinetic_grouped(counts1, x64, TAU, out=y64, workspace=ws64)
            torch.cuda.synchronize()
            f_steps = 2
            e0.record(stream)
            for _ in range(f_steps):
                p.kinetic_grouped(counts1, x64, TAU, out=y64, workspace=ws64)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / f_steps, ws64

        f_ms, ws64 = time_fp64(plan)   # FAST64 when the grid allows it
        x32 = x64.to(torch.complex64)
        y32 = torch.empty_like(x32)
        ws32 = torch.empty(plan.workspace_bytes(n1, torch.complex64), dtype=torch.uint8, device=dev)
        plan.kinetic_grouped(counts1, x32, TAU, out=y32, workspace=ws32)
        b64 = plan.forward_grouped(counts1, x64, workspace=ws64)
        b32 = plan.forward_grouped(counts1, x32, workspace=ws32)
        nrm = torch.linalg.vector_norm(x64, dim=1)
        err_rt = ((y32.to(torch.complex128) - y64).abs().amax(dim=1) / nrm).max().item()
        err_fw = ((b32.to(torch.complex128) - b64).abs().amax(dim=1) / nrm).max().item()
        drift = ((torch.linalg.vector_norm(b32.to(torch.complex128), dim=1) - nrm) / nrm).abs().max().item()
        del ws64, ws32, b64, b32
        fp64_value = 2 * n1 / (f_ms * 1e-3)
        dense_ms = None
        if rank == 0 and fast64 and args.workload == "precision":
            dplan = dsbt.Plan(N, R_MAX, L_MAX, fp64=True, tf32x3=False)   # dense FP64 T_l
            dense_ms, wsd = time_fp64(dplan)
            dplan.close()
            del wsd
            torch.cuda.empty_cache()
        if rank == 0:
            line["fp64_gpu"] = {"value": fp64_value, "unit": UNIT,
                                "scheme": "O(N l log N) FP64 (DSBT_PLAN_FAST64)" if fast64 else "dense FP64",
                                "sample": "batch 1 of the same workload (4096 complex128 channels)",
                                "ms_per_step": f_ms, "speedup_of_split_path": value / world / fp64_value,
                                "split_max_rel_err": {"kinetic_round_trip": err_rt, "forward": err_fw,
                                                      "norm_drift": drift}}
            if dense_ms is not None:
                line["fp64_gpu"]["dense_fp64"] = {"value": 2 * n1 / (dense_ms * 1e-3), "unit": UNIT,
                                                  "ms_per_step": dense_ms,
                                                  "speedup_of_split_path": value / world / (2 * n1 / (dense_ms * 1e-3))}

    # ---------------------------------------------------------- dense split-TF32 contraction (context)
    if rank == 0 and fast and args.workload == "precision":
        line["dense_tf32"] = dense_leg(dsbt, torch, counts, x, probes["tf32_tflops"], args)

    # ---------------------------------------------------------- TDSE (propagator + adjoint)
    if rank == 0 and not args.no_tdse and args.workload == "precision":
        line["tdse"] = tdse_leg(dsbt, inputs, torch, dev, probes["fp64_tflops"])

    # ---------------------------------------------------------- plain FP64 round trip (C2)
    if rank == 0 and not args.no_fp64 and args.workload == "precision":
        line["c2_fp64"] = c2_leg(dsbt, inputs, torch, dev)

    # ---------------------------------------------------------- uneven batch (one launch, graph)
    if rank == 0 and not args.no_batch and args.workload == "precision":
        plan.close()
        torch.cuda.empty_cache()
        dense_b = batch_leg(dsbt, inputs, torch, dev, max(3, args.steps // 3), 2, probes["tf32_tflops"], "dense")
        line["uneven_batch"] = batch_leg(dsbt, inputs, torch, dev, max(3, args.steps // 3), 2,
                                         probes["tf32_tflops"], "interval")
        line["uneven_batch"]["dense_persistent"] = dense_b

    # ---------------------------------------------------------- CPU oracle baseline
    if rank == 0 and world == 1 and not args.no_cpu:
        ntr, t_x, t_b, nt = oracle_sample()
        line["cpu_baseline"] = {"value": ntr / t_x, "unit": UNIT, "cores": nt, "kind": "oracle",
                                "sample": (f"{ntr} channel-transforms ({ntr // 4} complex channels each of l=1 and "
                                           f"l=2, N=4096, kinetic round trip by naive O(N^2) sums, {nt} threads, "
                                           f"one channel per call; the cost per channel is the same for every l, "
                                           f"so the rate stands for the whole workload); factor build for l=1,2 "
                                           f"{t_b:.1f} s excluded"),
                                "build_s_l12": t_b}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()   # idempotent
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
