#!/usr/bin/env python
"""Throughput of sigma = H C over the bosonic Fock basis (arXiv:2005.13679,
Eq. Haction) on GB300.

Default workload: generic Hermitian h/W, N = 100 bosons in M = 6 orbitals
(96,560,646 configurations, complex128 C of 1.5 GB, larger than L2), FP64-class
apply.  A step is one H C product with inputs resident in HBM.  Prints one JSON
line (rank 0).  Multi-GPU runs (torchrun) are independent replicas, one per
rank (weak scaling; the apply needs no exchange between replicas).

--impl reference times the plain CPU oracle (the only reference this project
has) on the host cores, on a bounded sample of rows of the same workload.
"""
from __future__ import annotations

import argparse
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

METRIC = "H·C applies/s and config-terms/s, FP64 vs FP32-mixed/batched, % of HBM roofline"
PREC = {"f64": 0, "f64_native": 1, "f32_mixed": 2}
DTYPE = {"f64": "f64 (fp32-pair arithmetic)", "f64_native": "f64", "f32_mixed": "c64 storage, fp32 products, fp32-pair accumulation"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws: int, local: int, backend: str = "nccl"):
    """Process group for N > 1 ranks (one per GPU, rendezvous from the
    MASTER_* environment); returns the barrier the timed region uses."""
    if ws == 1:
        return lambda: None
    import torch
    import torch.distributed as dist
    if backend == "nccl":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return lambda: dist.barrier()


def dist_reduce(x: float, op: str = "max") -> float:
    """x reduced over the ranks (max or sum); x itself for one rank."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.item()


def dist_finish() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


def shard(items, rank: int, ws: int) -> list:
    """Round-robin share of one rank: every item goes to exactly one rank."""
    return list(items)[rank::ws]


def batch_units(ws: int, per_rank: int = 64):
    """The independent Lieb-Liniger problems of the batch workload for ws ranks:
    per_rank * ws instances from one seeded stream (the first 64 are the
    single-GPU batch), each with its index in the stream (its state seed)."""
    from paper_2005_13679_gb300 import inputs
    return list(enumerate(inputs.uneven_ll_batch(count=per_rank * ws)))


# --------------------------------------------------------------------------
# CPU oracle timing (bounded sample of rows)
# --------------------------------------------------------------------------
def oracle_rate(w, h, W, C, seconds: float):
    import numpy as np

    import oracle
    oracle.build()
    rng = np.random.default_rng(123)
    n = 8
    while True:
        rows = rng.integers(0, w.nc, n)
        t0 = time.perf_counter()
        oracle.apply_rows(w.N, w.M, h, W, C, rows)
        dt = time.perf_counter() - t0
        if dt > 0.2 * seconds or n >= 1 << 22:
            break
        n = int(n * min(16.0, max(2.0, 0.3 * seconds / max(dt, 1e-4))))
    return n, dt


def host_info():
    """Host cores this process may use and the CPU model (lscpu, else the
    platform string)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": cores, "cpu_model": model}


def _oracle_worker(args):
    """One host core of the all-core oracle leg: attach the shared C, wait at
    the barrier, then evaluate `n` rows of sigma with the oracle's row form."""
    shm_name, nc, N, M, h, W, n, seed, barrier = args
    import numpy as np
    from multiprocessing import shared_memory

    import oracle
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        C = np.ndarray((nc,), dtype=np.complex128, buffer=shm.buf)
        rows = np.random.default_rng(seed).integers(0, nc, n)
        oracle.apply_rows(N, M, h, W, C, rows[: max(1, n // 50)])     # touch pages, load the library
        barrier.wait()
        t0 = time.perf_counter()
        oracle.apply_rows(N, M, h, W, C, rows)
        return time.perf_counter() - t0
    finally:
        del C
        shm.close()


def oracle_rate_all_cores(w, h, W, C, rows_per_core: int, cores: int):
    """The oracle as it stands on `cores` host processes at once (spawned, no
    CUDA context), each on its own bounded sample of rows: returns (rows in
    all, wall seconds of the slowest process)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np

    import oracle
    oracle.build()
    shm = shared_memory.SharedMemory(create=True, size=C.nbytes)
    try:
        np.ndarray(C.shape, dtype=np.complex128, buffer=shm.buf)[:] = C
        ctx = mp.get_context("spawn")
        with ctx.Manager() as mgr:
            bar = mgr.Barrier(cores)
            with ctx.Pool(cores) as pool:
                times = pool.map(_oracle_worker, [(shm.name, C.shape[0], w.N, w.M, h, W, rows_per_core, 1000 + i, bar)
                                                  for i in range(cores)])
        return rows_per_core * cores, max(times)
    finally:
        shm.close()
        shm.unlink()


def cpu_baseline(w, h, W, C, per_cfg: float, seconds: float, all_cores: bool = True):
    """cpu_baseline of the bench line: the oracle on one host core (bounded row
    sample, calibrated to ~seconds/5 .. seconds) and, when all_cores, on every
    host core at once (about the same work per core)."""
    info = host_info()
    n1, dt1 = oracle_rate(w, h, W, C, seconds)
    one = per_cfg * n1 / dt1
    out = {"value": one, "unit": "config-terms/s", "cores": 1, "kind": "oracle",
           "sample": f"{n1} random rows of sigma (row form), {dt1:.1f} s on one core", **info}
    if all_cores and info["nproc"] > 1:
        per_core = max(8, int(n1 * max(1.0, 0.5 * seconds / dt1)))
        nall, wall = oracle_rate_all_cores(w, h, W, C, per_core, info["nproc"])
        allc = per_cfg * nall / wall
        out.update({"value": allc, "cores": info["nproc"],
                    "sample": f"{nall} random rows of sigma (row form) on {info['nproc']} processes, "
                              f"{wall:.1f} s wall",
                    "single_core": {"value": one, "unit": "config-terms/s", "rows": n1, "seconds": dt1},
                    "parallel_speedup": allc / one})
    return out


def run_reference(args, w):
    """The oracle as it stands, on every host core: each step is one bounded
    sample of rows of sigma per core (all cores at once), timed on the host."""
    import numpy as np

    from paper_2005_13679_gb300 import inputs  # noqa: F401  (input generator only)
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    h, W = w.hamiltonian()
    C = w.state() if w.nrhs == 1 else w.state()[:, 0].copy()
    terms_total = terms_formula(w, h, W)
    per_cfg = terms_total / w.nc
    info = host_info()
    budget = max(3.0, min(30.0, 90.0 / max(1, args.steps + args.warmup)))
    rows_per_core, dt1 = oracle_rate(w, h, W, C, budget)
    for _ in range(args.warmup):
        oracle_rate_all_cores(w, h, W, C, max(1, rows_per_core // 8), info["nproc"])
    rows_all, wall = 0, 0.0
    for _ in range(args.steps):
        n, t = oracle_rate_all_cores(w, h, W, C, rows_per_core, info["nproc"])
        rows_all += n
        wall += t
    value = per_cfg * rows_all / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "config-terms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "M": w.M, "nc": w.nc},
        "cpu_baseline": {"value": value, "unit": "config-terms/s", "cores": info["nproc"], "kind": "oracle",
                         "sample": f"{rows_per_core} random rows of sigma per core per step (row form of the "
                                   f"oracle), {per_cfg:.1f} config-terms per configuration",
                         "single_core": {"value": per_cfg * rows_per_core / dt1, "unit": "config-terms/s"},
                         **info},
        "e2e": {"value": value, "unit": "config-terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# FP32 work of one executed term (one removal-addition pair of one
# configuration) for the path that runs, counting an FMA as 2 flop:
# * direct FP32-pair complex term: coefficient x amplitude (one packed pair
#   product, 14), two packed pair products with C (28) and two packed TwoSum
#   accumulations (28) = 70; real coefficients 35;
# * two-phase FP32-pair phase 1 (dense coefficients, M = 7, 8, or N beyond the
#   tensor-core layout): Gauss's three products, 1.5 packed pair products and
#   accumulations = 42;
# * FP32-mixed: direct 10 (real 6), two-phase 8 (two packed FMAs);
# * native FP64: 10 (real 6) on the FP64 pipe.
FLOPS_PER_TERM = {("f64", "direct"): 70, ("f64", "twophase"): 42, ("f32_mixed", "direct"): 10,
                  ("f32_mixed", "twophase"): 8, ("f64_native", "direct"): 10}
FLOPS_PER_TERM_REAL = {("f64", "direct"): 35, ("f32_mixed", "direct"): 6, ("f64_native", "direct"): 6}
# phase 1 of the pair-momentum form per (addition, (N-2)-configuration): the
# amplitude sqrt(n_s + 1) sqrt(n_l + 1 + d_sl) as an FP32-pair product (6), the
# factor o (2), the product with C (8) and the TwoSum accumulation (16); mixed:
# the amplitude (2) and one packed FMA (4)
PAIRS_FLOPS = {"f64": 32, "f32_mixed": 6}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12


def tc_shape(M):
    """Real-form sizes of the tensor-core phase 1 (fock_apply_tc.cuh): 2P real
    indices, the two MMA chains (N1 x K1 and N2 x K2), 20 digit pairs
    (levels i + j <= 7 with six digits of R and five of X)."""
    r2 = M * (M + 1)
    k1, k2 = (3 * r2 + 1 + 15) // 16 * 16, (2 * r2 + 15) // 16 * 16
    n2 = (3 * r2 + 1 + 15) // 16 * 16
    n1 = (n2 + 3 * r2 + 15) // 16 * 16
    return r2, n1 * k1 + n2 * k2, 20


def tc_shape_mixed(M):
    """Real-form sizes of the FP32-mixed tensor-core phase 1 (one chain N x K)
    and its 3 products (R_h X_h, R_h X_l, R_l X_h)."""
    r2 = M * (M + 1)
    return r2, ((r2 + 1 + 15) // 16 * 16) * ((3 * r2 + 1 + 15) // 16 * 16), 3


def nn_terms(w):
    """Terms the nearest-neighbour kernel evaluates: per configuration the
    diagonal and two hops per bond (M bonds on a ring, M = 2 has one)."""
    nb = w.M if w.M > 2 else 1
    return w.nc * (1 + 2 * nb)


def tc_flops(w, nnz_r, mixed=False):
    """Phase 1 per apply: the method's own work, one complex multiply-add
    (8 flop) per nonzero reduced coefficient per (N-2)-space column; the
    emulation's digit-pair products over the (2P)^2 real-form entries (2 flop
    each); and the MMA work executed (2 N K per column summed over the
    chains)."""
    r2, nk, pairs = tc_shape_mixed(w.M) if mixed else tc_shape(w.M)
    cols = math.comb(w.N - 2 + w.M - 1, w.M - 1) * w.nrhs
    return cols * 8 * nnz_r, cols * pairs * r2 * r2 * 2, cols * 2 * nk


def launches_per_step(path, prec):
    """Kernels of one apply: the FP32-pair input preparation (2), then the
    two-phase pair or one kernel."""
    return (2 if prec == 0 else 0) + (2 if path.startswith("twophase") else 1)


def reduced_nnz(w, h, W):
    """Nonzero reduced coefficients (removal multiset, addition multiset) with
    the one-body part folded in, as the library forms them."""
    import numpy as np
    M, N = w.M, w.N
    P = M * (M + 1) // 2
    idx = {}
    for k in range(M):
        for q in range(k, M):
            idx[(k, q)] = len(idx)
    R = np.zeros((P, P), dtype=np.complex128)
    for k in range(M):
        for q in range(M):
            for s in range(M):
                for l in range(M):
                    R[idx[(min(k, q), max(k, q))], idx[(min(s, l), max(s, l))]] += W[k, q, s, l]
                    if q == s:
                        R[idx[(min(k, q), max(k, q))], idx[(min(s, l), max(s, l))]] += h[k, l] / (N - 1)
    return int(np.count_nonzero(R))


def executed_terms(w, h, W):
    """Removal-addition pairs the kernel visits: each listed two-body pair is
    taken by the N_c(N-2, M) configurations that allow its removal (one-body:
    N_c(N-1, M))."""
    import numpy as np
    N, M = w.N, w.M
    nc = lambda n: math.comb(n + M - 1, M - 1) if n >= 0 else 0
    if W is None or N < 2:
        return nc(N - 1) * int(np.count_nonzero(h))
    return nc(N - 2) * reduced_nnz(w, h, W)


def sources_digest(paths):
    """First 16 hex digits of the SHA-256 of the listed source files (paths
    relative to the package directory), in the order given."""
    import hashlib
    pkg = os.path.join(ROOT, "paper_2005_13679_gb300")
    return hashlib.sha256(b"".join(open(os.path.join(pkg, f), "rb").read() for f in paths)).hexdigest()[:16]


def load_traffic(workload, precision, phase=""):
    """DRAM bytes per launch of the main kernel (phase="") or of the second
    phase of a two-phase apply (phase="_phase2") from the committed ncu summary
    of this workload, if the kernel's translation unit and the headers it
    includes (listed in the summary) still match the sources the counters were
    taken from (else None)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}_{precision}{phase}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        if sources_digest(vals["sources"].split()) != vals["sources_sha256_16"]:
            return None
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError, OSError):
        return None


def terms_formula(w, h, W):
    """Configuration terms of one apply (same definition as fock_hamiltonian_terms)."""
    import numpy as np
    N, M = w.N, w.M
    nc = lambda n: math.comb(n + M - 1, M - 1) if n >= 0 else 0
    P = M * (M + 1) // 2
    idx = {}
    for k in range(M):
        for q in range(k, M):
            idx[(k, q)] = len(idx)
    R = np.zeros((P, P), dtype=np.complex128)
    if W is not None:
        for k in range(M):
            for q in range(M):
                for s in range(M):
                    for l in range(M):
                        R[idx[(min(k, q), max(k, q))], idx[(min(s, l), max(s, l))]] += W[k, q, s, l]
    offh = int(np.count_nonzero(h - np.diag(np.diag(h))))
    return nc(N) + nc(N - 1) * offh + (nc(N - 2) * int(np.count_nonzero(R)) if N >= 2 else 0)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def time_steps(torch, fn, steps, warmup, barrier):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps


def run_sector(args, w):
    """One fixed-momentum sector of a Lieb-Liniger ring (weight sum_i i n_i =
    w.sector_Q): one step is one sector apply sigma = H C in the requested
    precision.  Also reports the other precisions, the end-to-end apply with
    host buffers, and the sector's Lanczos ground state."""
    import numpy as np
    import torch

    from paper_2005_13679_gb300 import fock
    ws, rank, local = dist_env()
    barrier = dist_init(ws, local)          # replicas: every rank the same sector
    if ws == 1:
        torch.cuda.set_device(0)
    fock.load()
    peaks, peak_src = load_peaks()
    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    sec = fock.Sector(sp, w.sector_Q)
    H = fock.Hamiltonian(sp, h, W)
    prec = PREC[args.precision]
    n = sec.size
    terms = fock.fock_sector_terms(sec.handle, H.handle)
    Cn = inputs_random_state(n, w.seed)
    Cd = torch.from_numpy(Cn).cuda()
    if prec == 2:
        Cd = Cd.to(torch.complex64)
    sig = torch.empty_like(Cd)
    wsb = torch.empty(max(fock.fock_sector_workspace_size(sec.handle, 1, prec), 16), dtype=torch.uint8,
                      device="cuda")
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in kev:
        a_.record(); b_.record()
    torch.cuda.synchronize()
    counter = {"i": -1}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # larger than L2

    def step():
        i = counter["i"]
        flush.zero_()
        fock.fock_apply_set_events(H.handle, *(kev[i] if 0 <= i < len(kev) else (None, None)))
        fock.fock_sector_apply_H(sec.handle, H.handle, Cd, sig, 1, prec, wsb)

    def step_timed():
        counter["i"] += 1
        step()

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        step()
    counter["i"] = -1
    ms = dist_reduce(time_steps(torch, step_timed, args.steps, 0, barrier), "max")
    clocks = clk.stop()
    fock.fock_apply_set_events(H.handle, None, None)
    kernel_ms = sum(a_.elapsed_time(b_) for a_, b_ in kev) / len(kev)
    elem = 8 if prec == 2 else 16
    nbytes = n * elem
    # end to end: pinned host C -> device, apply, device -> host
    Ch = torch.from_numpy(Cn).to(Cd.dtype).pin_memory()
    Sh = torch.empty_like(Ch).pin_memory()

    def e2e_step():
        Cd.copy_(Ch, non_blocking=True)
        fock.fock_sector_apply_H(sec.handle, H.handle, Cd, sig, 1, prec, wsb)
        Sh.copy_(sig, non_blocking=True)

    e2e_ms = time_steps(torch, e2e_step, max(3, args.steps // 2), 1, lambda: None)
    key = (args.precision, "direct")
    flops_term = FLOPS_PER_TERM_REAL[key] if H.real else FLOPS_PER_TERM[key]
    alu = terms * flops_term / (kernel_ms * 1e-3) / 1e12
    gbs = 2 * nbytes / (kernel_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": terms * ws / (ms * 1e-3), "unit": "config-terms/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "M": w.M, "sector_weight": w.sector_Q,
                   "total_momentum": w.sector_Q - w.N * (w.M // 2), "n_sector": n,
                   "nc_full": math.comb(w.N + w.M - 1, w.M - 1), "precision": args.precision,
                   "l2": "flushed before every step (256 MB write; the sector vectors fit L2)",
                   "parallelism": f"replicas x{ws}"},
        "sector_terms_per_apply": terms,
        "gpu_launches": (3 if prec == 0 else 1) * args.steps,
        "roofline": {"bound": "alu", "achieved": alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": alu / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "fock_sector_apply_kernel",
                     "kernel_ms": kernel_ms, "executed_terms": terms, "flops_per_term": flops_term,
                     "hbm_frac": gbs / peaks["hbm_gbs"], "peak_source": peak_src},
        "e2e": {"value": terms / (e2e_ms * 1e-3), "unit": "config-terms/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms},
        "clocks": clocks,
    }
    if args.extras:
        extras = {}
        for name, p in PREC.items():
            if p == prec:
                continue
            X = torch.from_numpy(Cn).cuda()
            if p == 2:
                X = X.to(torch.complex64)
            Y = torch.empty_like(X)
            wsx = torch.empty(max(fock.fock_sector_workspace_size(sec.handle, 1, p), 16), dtype=torch.uint8,
                              device="cuda")
            t = time_steps(torch, lambda: fock.fock_sector_apply_H(sec.handle, H.handle, X, Y, 1, p, wsx),
                           max(3, args.steps // 2), 1, lambda: None)
            extras[name] = {"ms_per_step": t, "config_terms_per_s": terms / (t * 1e-3)}
        out["other_precisions"] = extras
        t0 = time.perf_counter()
        E0, res, it, _, st = fock.fock_sector_lanczos_ground(sec.handle, H.handle, max_iter=args.lanczos_iters,
                                                             restart_len=30, tol=1e-10, seed=w.lanczos_seed)
        out["lanczos"] = {"seconds": time.perf_counter() - t0, "E0": E0, "residual": res, "products": it,
                          "status": int(st), "precision": "f64"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_finish()
    return 0


def inputs_random_state(n, seed):
    from paper_2005_13679_gb300 import inputs
    return inputs.random_state(n, seed)


def measure_one_by_one(torch, fock, probs, B, Cd, batch_ms):
    """The same FP64-class applies one instance at a time (each its own space,
    operator and the library's path for it, one workspace allocated
    beforehand), beside the batched apply."""
    objs = []
    for (N, M, h, W) in probs:
        sp = fock.Space(N, M)
        objs.append((sp, fock.Hamiltonian(sp, h, W)))
    sig = torch.empty_like(Cd)
    paths = {}
    # one workspace, the largest any instance prefers, shared by the sequence
    wsz = max(fock.fock_apply_workspace_size(sp.handle, H.handle, 1, fock.FOCK_PREC_F64) for sp, H in objs)
    wsb = torch.empty(max(wsz, 16), dtype=torch.uint8, device="cuda")

    def run():
        for i, (sp, H) in enumerate(objs):
            b, e = int(B.offsets[i]), int(B.offsets[i + 1])
            fock.fock_apply_H(sp.handle, H.handle, Cd[b:e], sig[b:e], 1, fock.FOCK_PREC_F64, fock.FOCK_ARM_AUTO, wsb)
    run()                                        # first launches
    for sp, H in objs:
        p = fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle, 1, fock.FOCK_PREC_F64, fock.FOCK_ARM_AUTO,
                                                 wsb.numel())]
        paths[p] = paths.get(p, 0) + 1
    t = time_steps(torch, run, 3, 1, lambda: None)
    ref = B.apply(Cd)
    err = float(torch.linalg.vector_norm(sig - ref) / torch.linalg.vector_norm(ref))
    del objs, sig, ref, wsb
    torch.cuda.empty_cache()
    return {"ms_per_step": t, "batched_ms": batch_ms, "workspace_bytes": wsz, "batched_speedup": t / batch_ms, "paths": paths,
            "rel_diff_vs_batched": err}


def batch_launches(B, prec):
    """Kernels of one batched apply: per instance with its own apply, the
    FP32-pair preparation (2, FP64-class) and the two phases; for the shared
    launch, the preparation of each of its instances (2 each, FP64-class) and
    the persistent kernel."""
    own = int(B.own.sum())
    shared = B.count - own
    prep = 2 if prec == 0 else 0
    return own * (prep + 2) + ((prep * shared + 1) if shared else 0)


def run_batch(args):
    """64 uneven Lieb-Liniger instances (N in [10, 200], M in 4..12, log g uniform,
    capped at 10^7 configurations each): one step is one batched FP64-class
    apply of every instance (its own two-phase apply for each instance of at
    least 2^18 configurations, one persistent launch with autotuned work items
    for the rest).  Also reports the FP32-mixed batched apply and the time to
    solve every ground state with the graph-captured batched Lanczos."""
    import tempfile

    import numpy as np
    import torch

    from paper_2005_13679_gb300 import fock, inputs
    ws, rank, local = dist_env()
    barrier = dist_init(ws, local)
    if ws == 1:
        torch.cuda.set_device(0)
    fock.load()
    # weak scaling: 64 independent problems per rank, dealt round-robin from
    # one seeded stream of 64 x ranks (no collective on the data path)
    mine = shard(batch_units(ws), rank, ws)
    inst = [x for _, x in mine]
    probs = [(x.N, x.M) + inputs.lieb_liniger_hw(x.M, x.g) for x in inst]
    B = fock.Batch(probs)
    C = np.empty(B.total, dtype=np.complex128)
    for i, (gi, _) in enumerate(mine):
        C[B.offsets[i]:B.offsets[i + 1]] = inputs.random_state(int(B.offsets[i + 1] - B.offsets[i]), 500 + gi)
    Cd = torch.from_numpy(C).cuda()
    sig = torch.empty_like(Cd)
    cache = os.path.join(tempfile.gettempdir(), "fock_batch_tune.txt")
    tiles, blocks = B.autotune(Cd, sig, fock.FOCK_PREC_F64, cache_path=cache)
    clk = ClockSampler(local)
    clk.start()
    ms = time_steps(torch, lambda: B.apply(Cd, sig, fock.FOCK_PREC_F64), args.steps, args.warmup, barrier)
    clocks = clk.stop()
    ms_all = dist_reduce(ms, "max")
    terms_all = dist_reduce(float(B.terms), "sum")
    out = {
        "metric": METRIC, "value": terms_all / (ms_all * 1e-3), "unit": "config-terms/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE["f64"], "data": "synthetic",
        "config": {"workload": "ll_batch64", "instances": B.count * ws, "instances_per_rank": B.count,
                   "total_nc_rank0": B.total,
                   "tiles_per_item": tiles, "blocks_per_sm": blocks, "l2": "inputs larger than L2 (no flush)"},
        "gpu_launches": batch_launches(B, fock.FOCK_PREC_F64) * args.steps, "clocks": clocks,
    }
    out["config"]["own_apply_instances"] = int(B.own.sum())
    if args.extras:
        out["one_by_one"] = measure_one_by_one(torch, fock, probs, B, Cd, ms_all)
        C32 = Cd.to(torch.complex64)
        s32 = torch.empty_like(C32)
        B.autotune(C32, s32, fock.FOCK_PREC_F32_MIXED, cache_path=cache)
        t32 = time_steps(torch, lambda: B.apply(C32, s32, fock.FOCK_PREC_F32_MIXED), args.steps, 2, lambda: None)
        out["other_precisions"] = {"f32_mixed": {"ms_per_step": t32, "config_terms_per_s": B.terms / (t32 * 1e-3)}}
        del C32, s32, Cd, sig
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        E, R, it, st = B.lanczos_ground(max_iter=args.lanczos_iters, restart_len=args.batch_restart, tol=1e-9,
                                        seed=11)
        dt = time.perf_counter() - t0
        out["lanczos"] = {"seconds": dt, "status": int(st), "products_max": int(it.max()),
                          "restart_len": args.batch_restart, "budget": args.lanczos_iters,
                          "products_mean": float(it.mean()), "max_rel_residual": float(np.max(R / np.abs(E))),
                          "converged": int(np.sum(R / np.abs(E) < 1e-6))}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_finish()
    return 0


def measure_separate(torch, fock, sp, H, Cn, w, steps):
    """The block of nrhs vectors in one apply against nrhs separate
    single-vector applies of the same operator (each column stored on its own),
    per precision: the block shares one decode and one set of targets and
    amplitudes per configuration."""
    res = {}
    for name in ("f64", "f32_mixed"):
        p = PREC[name]
        dt = torch.complex64 if p == 2 else torch.complex128
        blk = torch.from_numpy(Cn).to(dt).cuda()
        sblk = torch.empty_like(blk)
        wsb = torch.empty(max(fock.fock_apply_workspace_size(sp.handle, H.handle, w.nrhs, p), 16),
                          dtype=torch.uint8, device="cuda")
        t_blk = time_steps(torch, lambda: fock.fock_apply_H(sp.handle, H.handle, blk, sblk, w.nrhs, p,
                                                             fock.FOCK_ARM_AUTO, wsb), steps, 1, lambda: None)
        del wsb
        cols = [torch.from_numpy(Cn[:, j].copy()).to(dt).cuda() for j in range(w.nrhs)]
        outs = [torch.empty_like(c) for c in cols]
        ws1 = torch.empty(max(fock.fock_apply_workspace_size(sp.handle, H.handle, 1, p), 16), dtype=torch.uint8,
                          device="cuda")

        def sep():
            for c, o in zip(cols, outs):
                fock.fock_apply_H(sp.handle, H.handle, c, o, 1, p, fock.FOCK_ARM_AUTO, ws1)
        t_sep = time_steps(torch, sep, steps, 1, lambda: None)
        err = max(float(torch.linalg.vector_norm(outs[j] - sblk[:, j]) / torch.linalg.vector_norm(sblk[:, j]))
                  for j in range(w.nrhs))
        res[name] = {"block_ms": t_blk, "separate_ms": t_sep, "block_speedup": t_sep / t_blk,
                     "block_path": fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle, w.nrhs, p)],
                     "single_path": fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle, 1, p)],
                     "max_rel_diff_block_vs_single": err}
        del blk, sblk, cols, outs, ws1
        torch.cuda.empty_cache()
    return res


def measure_arms(torch, fock, sp, H, Cn, w, steps):
    """Jump-map tables (Sec. 4, Fig. 4) against the on-the-fly hash: build both
    maps, time the apply on the maps arm in each precision beside the hash arm,
    then free the maps."""
    import ctypes
    res = {}
    need = ctypes.c_size_t()
    fock.load().fock_build_jump_maps(sp.handle, 3, 1, ctypes.byref(need), fock._stream(None))
    res["map_bytes"] = need.value
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    vec = w.nc * w.nrhs * 16
    if need.value + 4 * vec > free:
        res["skipped"] = f"maps need {need.value / 1e9:.1f} GB, {free / 1e9:.1f} GB free"
        return res
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = fock.load().fock_build_jump_maps(sp.handle, 3, 0, None, fock._stream(None))
    torch.cuda.synchronize()
    res["build_s"] = time.perf_counter() - t0
    if st != 0:
        res["skipped"] = f"build failed: {fock.fock_strerror(st)}"
        return res
    try:
        for name, p in PREC.items():
            dt = torch.complex64 if p == 2 else torch.complex128
            X = torch.from_numpy(Cn).to(dt).cuda()
            Yh, Ym = torch.empty_like(X), torch.empty_like(X)
            wsb = torch.empty(max(fock.fock_apply_workspace_size(sp.handle, H.handle, w.nrhs, p), 16),
                              dtype=torch.uint8, device="cuda")
            row = {}
            for arm_name, arm, out in (("hash", fock.FOCK_ARM_HASH, Yh), ("maps", fock.FOCK_ARM_MAPS, Ym)):
                n = 1 if p == 1 else steps
                t = time_steps(torch, lambda: fock.fock_apply_H(sp.handle, H.handle, X, out, w.nrhs, p, arm, wsb),
                               n, 1, lambda: None)
                row[arm_name] = {"ms_per_step": t, "path": fock.PATH_NAMES[fock.fock_apply_path(
                    sp.handle, H.handle, w.nrhs, p, arm, wsb.numel())]}
            row["maps_over_hash_time"] = row["maps"]["ms_per_step"] / row["hash"]["ms_per_step"]
            row["max_rel_diff"] = float(torch.linalg.vector_norm(Ym - Yh) / torch.linalg.vector_norm(Yh))
            res[name] = row
            del X, Yh, Ym, wsb
            torch.cuda.empty_cache()
    finally:
        fock.load().fock_jump_maps_free(sp.handle)
    return res


def measure_lanczos_precision(torch, fock, sp, H, Cn, w, max_iter):
    """The precision form inside the Lanczos solver (Sec. 6): the FP32-mixed
    apply's error against the FP64-class apply on the workload's state, and
    the ground-state energy with mixed products (then FP64-class refinement)
    against FP64-class products throughout, each within max_iter products."""
    res = {}
    X = torch.from_numpy(Cn).cuda()
    ref = fock.fock_apply_H(sp.handle, H.handle, X, None, 1, fock.FOCK_PREC_F64)
    mixed = fock.fock_apply_H(sp.handle, H.handle, X.to(torch.complex64), None, 1, fock.FOCK_PREC_F32_MIXED)
    res["apply_rel_err_mixed_vs_f64"] = float(torch.linalg.vector_norm(mixed.to(torch.complex128) - ref)
                                              / torch.linalg.vector_norm(ref))
    del X, ref, mixed
    torch.cuda.empty_cache()
    runs = {}
    for name in ("f64", "f32_mixed"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E0, r, it, _, st = fock.fock_lanczos_ground(sp.handle, H.handle, max_iter=max_iter, restart_len=24,
                                                   tol=1e-10, seed=w.lanczos_seed, precision=PREC[name])
        runs[name] = {"E0": E0, "residual": r, "products": it, "status": int(st),
                      "seconds": time.perf_counter() - t0}
        torch.cuda.empty_cache()
    runs["rel_energy_diff_mixed_vs_f64"] = abs(runs["f32_mixed"]["E0"] - runs["f64"]["E0"]) / abs(runs["f64"]["E0"])
    res["lanczos"] = runs
    res["note"] = ("FP64 Krylov vectors and re-orthogonalisation; the mixed run switches to FP64-class products "
                   "at a relative residual of 1e-5 and ends with an FP64-class Rayleigh quotient")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="generic_n100_m6")
    ap.add_argument("--precision", default="f64", choices=list(PREC))
    ap.add_argument("--extras", type=int, default=1, help="also time the other precisions and forms")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-all-cores", type=int, default=1, help="also time the oracle on every host core")
    ap.add_argument("--e2e", type=int, default=1, help="also time the host-buffer entry point")
    ap.add_argument("--lanczos-iters", type=int, default=480, help="batched Lanczos budget (ll_batch64)")
    ap.add_argument("--batch-restart", type=int, default=16, help="batched Lanczos restart length (ll_batch64)")
    ap.add_argument("--arms", type=int, default=1, help="also time the jump-map arm (generic workloads)")
    ap.add_argument("--lanczos", type=int, default=1, help="Lanczos in both precisions (Lieb-Liniger workloads)")
    ap.add_argument("--lanczos-steps", type=int, default=200, help="product budget of that Lanczos run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2005_13679_gb300 import inputs
    if args.workload == "ll_batch64" and args.impl != "reference":
        return run_batch(args)
    w = inputs.WORKLOADS[args.workload]
    if w.sector_Q is not None:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "sector workloads have no oracle timing leg"}))
            return 0
        return run_sector(args, w)
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch

    from paper_2005_13679_gb300 import fock
    ws, rank, local = dist_env()
    barrier = dist_init(ws, local)
    if ws == 1:
        torch.cuda.set_device(0)
    fock.load()
    peaks, peak_src = load_peaks()

    h, W = w.hamiltonian()
    sp = fock.Space(w.N, w.M)
    H = fock.Hamiltonian(sp, h, W)
    prec = PREC[args.precision]
    Cn = w.state()
    Cd = torch.from_numpy(Cn).cuda()
    if prec == 2:
        Cd = Cd.to(torch.complex64)
    sig = torch.empty_like(Cd)
    wsz = fock.fock_apply_workspace_size(sp.handle, H.handle, w.nrhs, prec)
    wsb = torch.empty(max(wsz, 16), dtype=torch.uint8, device="cuda")

    # one event pair per timed step around the library's main kernel
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a_, b_ in kev:                      # materialise the CUDA events
        a_.record(); b_.record()
    torch.cuda.synchronize()
    counter = {"i": -1}

    def step():
        i = counter["i"]
        if 0 <= i < len(kev):
            fock.fock_apply_set_events(H.handle, kev[i][0], kev[i][1])
        else:
            fock.fock_apply_set_events(H.handle, None, None)
        fock.fock_apply_H(sp.handle, H.handle, Cd, sig, w.nrhs, prec, fock.FOCK_ARM_AUTO, wsb)

    def step_timed():
        counter["i"] += 1
        step()

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        step()
    counter["i"] = -1
    ms = time_steps(torch, step_timed, args.steps, 0, barrier)
    clocks = clk.stop()
    fock.fock_apply_set_events(H.handle, None, None)
    kernel_ms = sum(a_.elapsed_time(b_) for a_, b_ in kev) / len(kev)
    ms_all = dist_reduce(ms, "max")
    terms = H.terms * w.nrhs
    value = terms * ws / (ms_all * 1e-3)
    applies = ws * w.nrhs / (ms_all * 1e-3)

    # end to end through the host-buffer entry point (pinned buffers)
    elem = 8 if prec == 2 else 16
    Ch = (torch.from_numpy(Cn).to(torch.complex64) if prec == 2 else torch.from_numpy(Cn)).pin_memory()
    Sh = torch.empty_like(Ch).pin_memory()

    def e2e_step():
        fock.fock_apply_H_host(sp.handle, H.handle, Ch, Sh, w.nrhs, prec, fock.FOCK_ARM_AUTO)

    # each call is synchronous (copies in and out included): time the calls
    # one by one and report the median (host-side stalls of a shared machine
    # show up as outliers), with the mean and the minimum beside it
    e2e_ms, e2e_all = float("nan"), []
    if args.e2e:
        e2e_step()
        barrier()
        for _ in range(max(5, args.steps // 4)):
            t0 = time.perf_counter()
            e2e_step()
            e2e_all.append((time.perf_counter() - t0) * 1e3)
        barrier()
        e2e_ms = dist_reduce(sorted(e2e_all)[len(e2e_all) // 2], "max")
    del Ch, Sh

    nbytes = w.nc * w.nrhs * elem
    hbm_gbs = 2 * nbytes / (ms * 1e-3) / 1e9
    executed = executed_terms(w, h, W) * w.nrhs
    path = fock.PATH_NAMES[fock.fock_apply_path(sp.handle, H.handle, w.nrhs, prec, fock.FOCK_ARM_AUTO, wsz)]
    traffic = load_traffic(w.name, args.precision)
    if path == "twophase_tc":
        # dominant kernel = phase 1 on the tensor cores (fp16 digits, FP32
        # accumulators): the fraction is taken on the method's own flops; the
        # digit-pair work of the error-free split and the MMA work executed are
        # reported beside it
        nnz_r = reduced_nnz(w, h, W)
        alg, digit, mma = tc_flops(w, nnz_r, prec == 2)
        achieved = alg / (kernel_ms * 1e-3) / 1e12
        P = w.M * (w.M + 1) // 2
        ybytes = math.comb(w.N - 2 + w.M - 1, w.M - 1) * w.nrhs * P * (8 if prec == 2 else 16)
        traffic2 = load_traffic(w.name, args.precision, "_phase2")
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": achieved / peaks["bf16_tflops"], "traffic": traffic, "kernel": "fock_twophase_x_tc",
                    "kernel_ms": kernel_ms, "method_flops": alg,
                    "method_flops_note": "8 flop per nonzero reduced coefficient per (N-2)-space column",
                    "emulation": {"digit_pair_flops": digit, "executed_mma_flops": mma,
                                  "executed_tflops": mma / (kernel_ms * 1e-3) / 1e12,
                                  "executed_frac": mma / (kernel_ms * 1e-3) / 1e12 / peaks["bf16_tflops"]},
                    "hbm_frac_kernel": 2 * nbytes / (kernel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                    "hbm_frac_step": 2 * nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                    "hbm_note": "compulsory bytes of the apply (C read, sigma written) over the phase-1 and the "
                                "whole-step time",
                    "y_bytes_written": ybytes, "traffic_phase2": traffic2,
                    "traffic_apply": (traffic + traffic2) if (traffic and traffic2) else None,
                    "path": path,
                    "peak_note": "fp16 dense has the nominal bf16 rate on this part: measured bf16 burst "
                                 f"({peak_src}); of measured"}
    elif path == "nn":
        # one pass: C read once (neighbour reads hit L2), sigma written once;
        # the binding roof is the larger of the FP32-pipe and HBM fractions
        executed = nn_terms(w) * w.nrhs
        key = (args.precision, "direct")
        flops_term = FLOPS_PER_TERM_REAL[key] if H.real else FLOPS_PER_TERM[key]
        alu = executed * flops_term / (kernel_ms * 1e-3) / 1e12
        gbs = 2 * nbytes / (kernel_ms * 1e-3) / 1e9
        alu_frac, hbm_frac = alu / FP32_PEAK_TFLOPS, gbs / peaks["hbm_gbs"]
        if hbm_frac >= alu_frac:
            roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": hbm_frac, "traffic": traffic}
        else:
            roofline = {"bound": "alu", "achieved": alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": alu_frac, "traffic": traffic}
        roofline.update({"kernel": "fock_apply_nn", "kernel_ms": kernel_ms, "executed_terms": executed,
                         "flops_per_term": flops_term, "alu_frac": alu_frac, "hbm_frac": hbm_frac,
                         "algorithmic_bytes": 2 * nbytes, "path": path,
                         "peak_note": f"HBM: measured copy bandwidth ({peak_src}); FP32 pipe: 152 SMs x 128 "
                                      "lanes x 2 flop x 2070 MHz"})
    elif path == "twophase_block" and (H.forms & fock.FOCK_FORM_PAIR_MOMENTUM) and args.precision in PAIRS_FLOPS:
        # phase 1 of the pair-momentum form: one amplitude-times-C product per
        # (addition pair, (N-2)-configuration), no coefficient products
        P = w.M * (w.M + 1) // 2
        executed = math.comb(w.N - 2 + w.M - 1, w.M - 1) * P * w.nrhs
        flops_term = PAIRS_FLOPS[args.precision]
        achieved = executed * flops_term / (kernel_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                    "kernel": "phase 1 (pair-momentum amplitudes Z_K)", "kernel_ms": kernel_ms,
                    "executed_terms": executed, "flops_per_term": flops_term, "path": path,
                    "form": "pair_momentum",
                    "z_bytes_written": math.comb(w.N - 2 + w.M - 1, w.M - 1) * w.nrhs * (2 * w.M - 1)
                                       * (8 if prec == 2 else 16),
                    "traffic_phase2": load_traffic(w.name, args.precision, "_phase2"),
                    "pipe": "FP32 (fma.rn.f32x2 and scalar); peak = 152 SMs x 128 lanes x 2 flop x 2070 MHz"}
    else:
        key = (args.precision, "twophase" if path.startswith("twophase") else "direct")
        flops_term = FLOPS_PER_TERM_REAL[key] if (H.real and key in FLOPS_PER_TERM_REAL) else FLOPS_PER_TERM[key]
        achieved = executed * flops_term / (kernel_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                    "kernel": "phase 1" if path.startswith("twophase") else "main",
                    "kernel_ms": kernel_ms, "executed_terms": executed, "flops_per_term": flops_term,
                    "path": path,
                    "pipe": "FP32 (fma.rn.f32x2 and scalar); peak = 152 SMs x 128 lanes x 2 flop x 2070 MHz"}
    out = {
        "metric": METRIC, "value": value, "unit": "config-terms/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "M": w.M, "nc": w.nc, "nrhs": w.nrhs,
                   "precision": args.precision, "arm": "hash", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws}"},
        "applies_per_s": applies,
        "config_terms_per_apply": terms,
        "gpu_launches": launches_per_step(path, prec) * args.steps,
        "roofline": roofline,
        "hbm": {"compulsory_bytes": 2 * nbytes, "achieved_gbs": hbm_gbs, "peak_gbs": peaks["hbm_gbs"],
                "frac": hbm_gbs / peaks["hbm_gbs"], "peak_source": peak_src},
        "e2e": {"value": terms * ws / (e2e_ms * 1e-3), "unit": "config-terms/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms,
                "statistic": "median of per-call host times",
                "mean_ms": sum(e2e_all) / len(e2e_all) if e2e_all else None,
                "min_ms": min(e2e_all) if e2e_all else None, "calls": len(e2e_all)},
        "clocks": clocks,
    }
    if rank == 0 and args.extras:
        extras = {}
        for name, p in PREC.items():
            if p == prec:
                continue
            X = torch.from_numpy(Cn).cuda()
            if p == 2:
                X = X.to(torch.complex64)
            Y = torch.empty_like(X)
            del wsb                                  # each precision gets its own preferred workspace
            wsb = torch.empty(max(fock.fock_apply_workspace_size(sp.handle, H.handle, w.nrhs, p), 16),
                              dtype=torch.uint8, device="cuda")
            steps = 2 if p == 1 else max(3, args.steps // 2)
            t = time_steps(torch, lambda: fock.fock_apply_H(sp.handle, H.handle, X, Y, w.nrhs, p,
                                                              fock.FOCK_ARM_AUTO, wsb), steps, 1, lambda: None)
            extras[name] = {"ms_per_step": t, "config_terms_per_s": terms / (t * 1e-3)}
            del X, Y
        out["other_precisions"] = extras
        del wsb
        torch.cuda.empty_cache()
        if w.nrhs > 1:
            out["separate_applies"] = measure_separate(torch, fock, sp, H, Cn, w, max(3, args.steps // 4))
        if args.arms and w.kind != "ll":
            out["arms"] = measure_arms(torch, fock, sp, H, Cn, w, max(2, args.steps // 8))
        if args.lanczos and w.kind == "ll":
            out["lanczos_precision"] = measure_lanczos_precision(torch, fock, sp, H, Cn, w, args.lanczos_steps)
        if w.nrhs == 1 and w.M <= 12:
            # one- and two-body density matrices of the same state (Eqs. rho1, rho2)
            X = torch.from_numpy(Cn).cuda()
            fock.fock_density_matrices(sp.handle, X, w.M)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                fock.fock_density_matrices(sp.handle, X, w.M)
            t = (time.perf_counter() - t0) / reps * 1e3
            fock.fock_density_matrices(sp.handle, X, w.M, want_rho2=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fock.fock_density_matrices(sp.handle, X, w.M, want_rho2=False)
            t1 = (time.perf_counter() - t0) / reps * 1e3
            P = w.M * (w.M + 1) // 2
            out["density_matrices"] = {
                "ms_per_call": t, "rho1_only_ms_per_call": t1,
                "rho1_columns": math.comb(w.N - 1 + w.M - 1, w.M - 1),
                "rho2_columns": math.comb(w.N - 2 + w.M - 1, w.M - 1) if w.N >= 2 else 0,
                "rho2_gram_entries": P * (P + 1) // 2,
                "note": "host-synchronous calls incl. the input split (the workspace is kept with the space "
                        "after the first call); rho2 is a Gram matrix over the (N-2)-particle space and rho1 "
                        "its partial trace; alone, rho1 is a Gram matrix over the (N-1)-particle space"}
            del X
        out["cpu_baseline"] = cpu_baseline(w, h, W, Cn if w.nrhs == 1 else Cn[:, 0].copy(), H.terms / w.nc,
                                           args.cpu_seconds, all_cores=bool(args.cpu_all_cores))
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist_finish()
    return 0


if __name__ == "__main__":
    sys.exit(main())
