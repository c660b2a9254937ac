#!/usr/bin/env python
"""Benchmark: RIXS map throughput (incident x loss energy points per second).

One step = one whole RIXS map of the workload (Eqs. 1-2): Hubbard operators,
FP64 Lanczos ground state, the multi-shifted BiCG solve for every incident
energy, the sector maps and the batched continued fraction of the second step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` times msb_rixs_map_ops (operators
built beforehand, map left on the device) with CUDA events on the calling
stream, with the library profiler off (the solve replays its CUDA graphs).
One more map with the profiler on (every launch bracketed by CUDA events on
its stream) gives the kernel shares and the dominant kernel's roofline.
`e2e` times msb_rixs_map (host grids in, host map out, operators built inside
the call) with a wall clock.  For the default FP32-mixed L = 14 workload the
line adds `precision_comparison`: the same map once in the plain FP64 form
(speed-up and relative L2 difference).  Under torchrun each rank computes the
map of its own core site (independent problems, no collective on the data
path): weak scaling.

Workloads (--workload): hubbard-L14-mixed (default: L = 14, 201 x 400 points,
FP32 vectors and apply, FP64 scalars), hubbard-L14-fp64, hubbard-L12-fp64,
hubbard-L8-fp64, hubbard-L12x12rhs-mixed (one right-hand side per core site,
one joint solve), hubbard-L10-11-12-clusters-mixed (three clusters of uneven
size in one solve and one continued fraction; its line adds `separate_maps`),
hubbard-L12-q12-mixed (momentum-resolved maps over the 12 core sites),
random-csr-fp64 and random-csr-mixed (n = 2^22, 256 shifts; one step = the
multi-shift solve), solve-sweep-L12 (Fig. 4: MSBiCG vs per-energy BiCGStab,
MVMs, seconds and memory against the number of incident energies) and
cf-tolerance-study (map error against the continued fraction's stopping rule).

`cpu_baseline`: the oracle on the host cores (a process pool, the core count
from the affinity mask): the whole map for small workloads, and for L = 12 / 14
a bounded, labelled sample (the oracle's build of H and H' and its sparse
products timed with every core busy) scaled with the oracle's own per-row
counts.  The default line also carries the oracle's whole L = 8 map timed on
all cores (`cpu_full_small_map`).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

# name -> (workload, precision, solve_tol, cf_tol).  The continued-fraction tolerance is
# the loosest that keeps the map within its bar with a margin: the map's error against
# the converged fraction is about 0.4 cf_tol (FP64: 1e-9 -> 4e-10 against the 1e-8 bar;
# FP32-mixed: 1e-5 -> 4e-6 to 6e-6 against the 1e-4 bar).
WORKLOADS = {
    "hubbard-L12-fp64": (workloads.CHAIN12, 0, 1e-10, 1e-9),
    "hubbard-L14-mixed": (workloads.CHAIN14, 1, 1e-8, 1e-5),
    "hubbard-L14-fp64": (workloads.CHAIN14, 0, 1e-10, 1e-9),
    "hubbard-L8-fp64": (workloads.CHAIN8, 0, 1e-10, 1e-9),
    "hubbard-L12x12rhs-mixed": (workloads.BATCH_SITES, 1, 1e-8, 1e-5),
    "hubbard-L12-q12-mixed": (workloads.BATCH_SITES, 1, 1e-8, 1e-5),
}
# workloads with one right-hand side per core site (one call, one shared second step)
SITES = {"hubbard-L12x12rhs-mixed": list(range(12))}
# momentum-resolved maps (coherent sum over all core sites): name -> number of momenta 2 pi k / L
QMAPS = {"hubbard-L12-q12-mixed": 12}
# clusters of uneven size in one call: name -> (clusters, precision, solve_tol, cf_tol)
CLUSTERS = {"hubbard-L10-11-12-clusters-mixed": (workloads.BATCH_CLUSTERS, 1, 1e-8, 1e-5)}
# the precision comparison: an FP32-mixed workload -> its FP64 form, run once on the same model
FP64_FORM = {"hubbard-L14-mixed": "hubbard-L14-fp64"}
DEFAULT = "hubbard-L14-mixed"
# the solve-cost sweep of Fig. 4 (MSBiCG vs per-energy BiCGStab on the GPU)
SWEEP = "solve-sweep-L12"
# the continued fraction's stopping rule against the map error
CF_STUDY = "cf-tolerance-study"
SWEEP_N_IN = (10, 30, 100, 300)
# random complex-symmetric stress workload: name -> precision, tolerance
CSR_WORKLOADS = {"random-csr-fp64": (0, 1e-10), "random-csr-mixed": (1, 1e-7)}

# Roofline denominators.  HBM: the measured copy bandwidth of this machine.  FP64: the
# nominal GB300 FP64 rate of the profiling recipe, 1.25 TFLOP/s (not measured).
FP64_PEAK_TFLOPS = 1.25


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        if self.gpu is None:
            return self
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.path is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (--no-clocks)"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            lines = open(self.path).read().strip().splitlines()
        except OSError:
            lines = []
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if self.path:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on all host cores
# ---------------------------------------------------------------------------
def oracle_costs(name: str):
    path = os.path.join(ROOT, "profiles", f"oracle_costs_{name}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _oracle_pool(n_jobs: int):
    """Spawn pool (this process holds a CUDA context) of single-threaded workers."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    os.environ["CUDA_VISIBLE_DEVICES"] = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return mp.get_context("spawn").Pool(max(1, min(n_jobs, host_cores())))


def _oracle_row(job):
    """One row of the map by the oracle's plain definition (independent BiCGStab to
    1e-13, continued fraction to 1e-13); returns its intensity row and seconds."""
    import scipy.sparse as sp
    from oracle import hubbard, solvers, spectrum
    L, n_up, n_dn, core, Gamma, eta, E_G, G, w_in, w = job
    t0 = time.perf_counter()
    gsec, isec = hubbard.Sector(L, n_up, n_dn), hubbard.Sector(L, n_up + 1, n_dn)
    H = hubbard.hamiltonian_kron(gsec, 1.0, 8.0)
    Hp = hubbard.hamiltonian_kron(isec, 1.0, 8.0, 4.0, core)
    O2 = hubbard.creation_operator(gsec, isec, core, 0)
    O1 = hubbard.annihilation_operator(isec, gsec, core, 0)
    A = (Hp - (E_G + w_in + 1j * Gamma) * sp.identity(Hp.shape[0], format="csr")).tocsr()
    psi, _ = solvers.bicgstab(lambda v: A @ v, (O2 @ G).astype(np.complex128), 1e-13)
    I, _ = spectrum.lanczos_cf(H, O1 @ psi, E_G, np.asarray(w), eta, cf_tol=1e-13)
    return I, time.perf_counter() - t0


def cpu_full_map(wl, return_map: bool = False) -> dict:
    """The oracle's whole map of a small workload, rows spread over all host cores
    (wall clock: build + ground state in this process, then the rows in a pool)."""
    from oracle import hubbard, solvers
    t0 = time.perf_counter()
    H = hubbard.hamiltonian_kron(hubbard.Sector(wl.L, wl.n_up, wl.n_dn), 1.0, 8.0)
    E_G, G, _ = solvers.ground_state(H, workloads.lanczos_start(H.shape[0], wl.lanczos_seed))
    jobs = [(wl.L, wl.n_up, wl.n_dn, wl.core_site, wl.Gamma, wl.eta, E_G, G, float(x), wl.w) for x in wl.w_in]
    with _oracle_pool(len(jobs)) as pool:
        rows = pool.map(_oracle_row, jobs)
    sec = time.perf_counter() - t0
    pts = wl.n_in * wl.n_w
    out = {"workload": wl.name, "value": pts / sec, "unit": "map points/s", "seconds": sec,
           "cores": min(len(jobs), host_cores()), "kind": "oracle",
           "sample": f"the whole {wl.n_in} x {wl.n_w} map of {wl.name}, one row per worker process"}
    if return_map:
        out["map"] = np.array([r[0] for r in rows])
        out["E_G"] = E_G
    return out


def _spmv_worker(job):
    """k complex SpMVs with each of the memory-mapped matrices; seconds per product."""
    import scipy.sparse as sp
    d, names, k = job
    out = {}
    for nm in names:
        rowptr = np.load(os.path.join(d, nm + "_rowptr.npy"), mmap_mode="r")
        col = np.load(os.path.join(d, nm + "_col.npy"), mmap_mode="r")
        val = np.load(os.path.join(d, nm + "_val.npy"), mmap_mode="r")
        n = len(rowptr) - 1
        A = sp.csr_matrix((val, col, rowptr), shape=(n, n), copy=False)
        x = np.random.default_rng(1).standard_normal(n) + 0j
        A @ x
        t0 = time.perf_counter()
        for _ in range(k):
            x = A @ x
            x /= np.abs(x).max()
        out[nm] = (time.perf_counter() - t0) / k
    return out


def _build_worker(job):
    """Build H and H' of a workload with the oracle (Kronecker assembly) and store
    their CSR arrays in directory d; returns the build seconds."""
    from oracle import hubbard
    d, L, n_up, n_dn, core = job
    t0 = time.perf_counter()
    H = hubbard.hamiltonian_kron(hubbard.Sector(L, n_up, n_dn), 1.0, 8.0)
    Hp = hubbard.hamiltonian_kron(hubbard.Sector(L, n_up + 1, n_dn), 1.0, 8.0, 4.0, core)
    sec = time.perf_counter() - t0
    for nm, M in (("H", H), ("Hp", Hp)):
        np.save(os.path.join(d, nm + "_rowptr.npy"), M.indptr.astype(np.int64))
        np.save(os.path.join(d, nm + "_col.npy"), M.indices.astype(np.int32))
        np.save(os.path.join(d, nm + "_val.npy"), M.data)
    return sec


def cpu_sampled_map(name: str, wl) -> dict:
    """A bounded sample of the oracle on a large workload, scaled to the whole map.

    Measured: the oracle's build of H and H' (one process), and the throughput of
    complex sparse products of H and of H' with every host core busy (one worker
    per core, each running its own products on memory-mapped copies).  Scaled:
    whole map = build + ground state (gs products of H on one core) + n_in rows x
    (BiCGStab products of H' + continued-fraction products of H) spread over all
    cores, with the oracle's own per-row counts measured in full on the L = 12
    workload (profiles/oracle_costs_hubbard-L12-fp64.json)."""
    costs = oracle_costs("hubbard-L12-fp64")
    if costs is None:
        return {"value": None, "unit": "map points/s", "cores": host_cores(), "kind": "oracle",
                "sample": "not sampled: no recorded per-row oracle counts"}
    P = host_cores()
    need = 2.2 * 16 * math.comb(wl.L, wl.n_up) * math.comb(wl.L, wl.n_dn) * 12     # both CSR matrices, with margin
    base = None
    for cand in ("/dev/shm", tempfile.gettempdir()):
        try:
            if os.path.isdir(cand) and shutil.disk_usage(cand).free > need:
                base = cand
                break
        except OSError:
            continue
    if base is None:
        return {"value": None, "unit": "map points/s", "cores": P, "kind": "oracle",
                "sample": "not sampled: no scratch directory with room for the oracle's H and H'"}
    with tempfile.TemporaryDirectory(dir=base) as d:
        with _oracle_pool(1) as pool:
            t_build = pool.apply(_build_worker, ((d, wl.L, wl.n_up, wl.n_dn, wl.core_site),))
        k = 4
        with _oracle_pool(P) as pool:
            t0 = time.perf_counter()
            res = pool.map(_spmv_worker, [(d, ("H", "Hp"), k)] * P)
            t_pool = time.perf_counter() - t0
    t_H = statistics.median(r["H"] for r in res)          # seconds per product, all cores busy
    t_Hp = statistics.median(r["Hp"] for r in res)
    gs = costs["ground_state_matvecs"]
    mv_row, depth_row = costs["mean_solve_matvecs"], costs["mean_cf_depth"]
    T_rows = wl.n_in * (mv_row * t_Hp + depth_row * t_H) / P
    T_map = t_build + gs * t_H + T_rows
    pts = wl.n_in * wl.n_w
    return {"value": pts / T_map, "unit": "map points/s", "cores": P, "kind": "oracle",
            "sample": (f"oracle (numpy/scipy) on {name}: build of H and H' measured ({t_build:.1f} s, one process); "
                       f"complex sparse products measured with {P} worker processes busy at once "
                       f"({t_H * 1e3:.0f} ms per H product, {t_Hp * 1e3:.0f} ms per H' product, {k} of each per "
                       f"worker, {t_pool:.1f} s); whole map = build + {gs} ground-state products + {wl.n_in} rows x "
                       f"({mv_row:.0f} BiCGStab products of H' + {depth_row:.0f} continued-fraction products of H) "
                       f"over {P} cores, the per-row counts being the oracle's own, measured in full on "
                       f"hubbard-L12-fp64 (an estimate, labelled as such)"),
            "seconds_measured": t_build + t_pool, "map_seconds_estimated": T_map, "estimate": True}


# Workloads whose oracle map runs in full within the baseline's bound; larger single-map
# workloads get the sampled estimate.
ORACLE_FULL_MAX_DIM = 20_000


def run_cpu_baseline(name: str) -> dict:
    try:
        return _run_cpu_baseline(name)
    except Exception as e:                       # the baseline never stops the GPU line
        return {"value": None, "unit": "map points/s", "cores": host_cores(), "kind": "oracle",
                "sample": f"failed: {type(e).__name__}: {e}"}


def _run_cpu_baseline(name: str) -> dict:
    if name not in WORKLOADS:
        return {"value": None, "unit": "map points/s", "cores": host_cores(), "kind": "oracle",
                "sample": f"not sampled for the batch workload {name}"}
    wl = WORKLOADS[name][0]
    if math.comb(wl.L, wl.n_up) * math.comb(wl.L, wl.n_dn) <= ORACLE_FULL_MAX_DIM:
        return cpu_full_map(wl)
    return cpu_sampled_map(name, wl)


# ---------------------------------------------------------------------------
# Multi-rank logic: independent problems per rank, no collective on the data path
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the whole job's time is the slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_core_site(rank: int, L: int) -> int:
    """The core-hole site whose map this rank computes (translation-equivalent problems)."""
    return rank % L


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measured_traffic(workload, kernel, alg_bytes_per_launch, shape=None):
    """DRAM bytes per launch scaled from an ncu capture of the same kernel (None if none,
    or if the capture was of another launch shape than the one that ran)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[workload][kernel]
    except (OSError, KeyError, ValueError):
        return None
    if shape is not None and rec.get("shape") not in (None, shape):
        return None
    return rec["dram_bytes"] / rec["alg_bytes"] * alg_bytes_per_launch


def dominant_roofline(stats, prec, peaks, workload=None, shape=None):
    top = max(stats, key=lambda s: s["ms"])
    avg_ms = top["ms"] / top["launches"]
    traffic = measured_traffic(workload, top["name"], top["alg_bytes"] / top["launches"], shape)
    if prec == 0 and top["name"] != "cf_apply":
        # FP64 complex multiply-adds per shift (the per-shift update): FP64-pipe bound
        achieved = top["alg_flops"] / top["launches"] / (avg_ms * 1e-3) / 1e12
        return top, {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": top["name"],
                     "peak_source": "nominal FP64 rate, 1.25 TFLOP/s (not measured)"}
    # The Hamiltonian apply is a streaming sparse operation: its roofline is HBM in both
    # precisions (in FP64 the hop sums are integer fixed point; the FP64 pipe does the
    # diagonal, the V_{k-1} term, the conversion and the product, 10 operations per element).
    achieved = top["alg_bytes"] / top["launches"] / (avg_ms * 1e-3) / 1e9
    return top, {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": top["name"],
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}


def gpu_arm_csr(args, rank, world):
    """n = 2^22 random real symmetric matrix, 256 shifts sigma_k + 0.3i: one step =
    the multi-shift solve of all shifts (solutions stay on the device)."""
    import torch
    from paper_2506_09551_gb300 import api, native

    native.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    prec, tol = CSR_WORKLOADS[args.workload]
    wl = workloads.RANDOM_CSR
    rowptr, col, val = workloads.random_symmetric_csr(wl.n, wl.half_nnz_per_row, wl.diag_range,
                                                      wl.matrix_seed + rank)
    b = torch.tensor(workloads.random_complex_rhs(wl.n, wl.rhs_seed + rank), device="cuda")
    sig = workloads.random_shifts(wl.n_shifts, *wl.shift_range, wl.shift_imag, wl.shift_seed)
    seed = int(np.argsort(sig.real)[len(sig) // 2])
    op = api.Operator.csr(rowptr, col, val)
    lib = native.load()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step():
        return op.multishift_solve(b, sig - sig[seed], -sig[seed], tol=tol, maxit=20000, prec=prec,
                                   allow_status=(native.MSB_EMAXITER,))

    x = None
    for _ in range(args.warmup):
        del x
        x, per, info, st = step()
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None if args.no_clocks else str(local)) as clk:
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            del x
            x, per, info, st = step()
        e1.record(stream)
        e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    # one more step with the library profiler on, for the kernel shares and the roofline
    del x
    lib.msb_profile_reset()
    lib.msb_profile_enable(1)
    x, per, info_p, st = step()
    torch.cuda.synchronize()
    lib.msb_profile_enable(0)
    stats = native.profile_read()
    del x
    # end to end: host matrix and right-hand side in, host solutions out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if not args.no_e2e:
        op2 = api.Operator.csr(rowptr, col, val)
        b2 = torch.tensor(workloads.random_complex_rhs(wl.n, wl.rhs_seed + rank)).pin_memory().to("cuda")
        x2, *_ = op2.multishift_solve(b2, sig - sig[seed], -sig[seed], tol=tol, maxit=20000, prec=prec,
                                      allow_status=(native.MSB_EMAXITER,))
        xh = x2.cpu()
        del op2, x2, xh
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    top, roof = dominant_roofline(stats, prec, measured_peaks())
    total_ms = sum(s_["ms"] for s_ in stats)
    csz = 16 if prec == 0 else 8
    return {
        "metric": "shifted solves/s (random complex-symmetric CSR)",
        "value": job_throughput(wl.n_shifts, world, ms * 1e-3),
        "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if prec == 0 else "c64 vectors, f64 scalars", "data": "synthetic random CSR",
        "config": {"workload": args.workload, "n": wl.n, "nnz": int(len(val)), "n_shifts": wl.n_shifts,
                   "tol": tol, "seed_shift": seed, "l2": "working set larger than L2; no flush needed"},
        "e2e": {"value": job_throughput(wl.n_shifts, world, e2e_s), "unit": "solves/s",
                "h2d_bytes_per_step": int(rowptr.nbytes + col.nbytes + val.nbytes + wl.n * 16),
                "d2h_bytes_per_step": int(wl.n_shifts * wl.n * csz), "seconds": e2e_s},
        "gpu_launches": int(info["kernel_launches"]),
        "roofline": roof, "clocks": clk.summary(),
        "profiled_step": "kernel shares and roofline from one extra solve with the library profiler on",
        "solve": {"iterations": info["iterations"], "n_converged": info["n_converged"],
                  "max_shift_residual": info["max_shift_residual"], "device_bytes": info["device_bytes"]},
        "kernels": sorted([{"name": s_["name"], "launches": s_["launches"], "ms": round(s_["ms"], 3),
                            "share": round(s_["ms"] / total_ms, 4)} for s_ in stats], key=lambda d: -d["ms"]),
        "cpu_baseline": None,
    }


def gpu_arm_sweep(args, rank, world):
    """The paper's cost comparison (Sec. III, Fig. 4) on the GPU: the solves of Eq. 2 for
    n_w_in incident energies on [-4, 12] of the L = 12 ring, by the multi-shifted BiCG
    (one Krylov space for all) and by per-energy BiCGStab (one each), both FP64 to
    tolerance 1e-10: operator products, device seconds and device memory per n_w_in."""
    import torch
    from paper_2506_09551_gb300 import api, native

    native.load()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = workloads.CHAIN12
    m = api.model(wl.L, wl.n_up, wl.n_dn)
    H = api.Operator.hubbard(m, False)
    Hp = api.Operator.hubbard(m, True)
    E_G, G, _ = H.ground_state(wl.gs_tol, 300)
    b = api.apply_cdag_up(m, 0, G.to(torch.complex128), Hp.dim)
    stream = torch.cuda.current_stream()
    rows = []
    for n_in in SWEEP_N_IN:
        w_in = np.linspace(wl.w_in_range[0], wl.w_in_range[1], n_in)
        seed = workloads.seed_index(w_in)
        c0 = -(E_G + 1j * wl.Gamma)
        rec = {"n_w_in": n_in}
        for name, run in (("msbicg", lambda: Hp.multishift_solve(b, w_in - w_in[seed], c0=c0 - w_in[seed],
                                                                  tol=1e-10, maxit=20000,
                                                                  allow_status=(native.MSB_EMAXITER,))),
                          ("bicgstab", lambda: Hp.bicgstab(b, w_in, c0=c0, tol=1e-10, maxit=20000))):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, per, info, st = run()
            e1.record(stream)
            e1.synchronize()
            rec[name] = {"seconds": e0.elapsed_time(e1) * 1e-3, "matvecs": int(info["matvecs"]),
                         "iterations": int(info["iterations"]), "n_converged": int(info["n_converged"]),
                         "device_bytes": int(info["device_bytes"]) + int(x.numel() * x.element_size())}
            if name == "msbicg":
                xm = x
            else:
                rec["max_rel_diff"] = float((torch.linalg.vector_norm(x - xm, dim=1) /
                                             torch.linalg.vector_norm(xm, dim=1)).max().item())
            del x
        del xm
        rec["speedup"] = rec["bicgstab"]["seconds"] / rec["msbicg"]["seconds"]
        rec["matvec_ratio"] = rec["bicgstab"]["matvecs"] / max(rec["msbicg"]["matvecs"], 1)
        rows.append(rec)
        print(f"[bench] sweep n_w_in={n_in}: MSBiCG {rec['msbicg']['seconds']:.2f} s / {rec['msbicg']['matvecs']} "
              f"MVMs, BiCGStab {rec['bicgstab']['seconds']:.2f} s / {rec['bicgstab']['matvecs']} MVMs",
              file=sys.stderr, flush=True)
    return {"metric": "Eq. 2 solves: MSBiCG vs per-energy BiCGStab (Fig. 4)", "unit": "seconds, MVMs, bytes",
            "value": rows[-1]["speedup"], "value_is": f"speed-up at n_w_in = {rows[-1]['n_w_in']}",
            "n_gpus": 1, "dtype": "c128", "data": "synthetic: L = 12 Hubbard ring, GPU ground state",
            "config": {"workload": args.workload, "L": wl.L, "dim_intermediate": int(Hp.dim), "tol": 1e-10,
                       "Gamma": wl.Gamma, "w_in_range": list(wl.w_in_range)},
            "sweep": rows}


def gpu_arm_cf_study(args, rank, world):
    """The continued fraction's stopping rule against accuracy: maps of the L = 12
    workload (all 101 x 400 points) and of 21 incident energies of the L = 14 workload at
    several cf_tol, each against the same map with a converged fraction (FP64, cf_tol
    1e-13 at L = 12, 1e-11 at L = 14): relative L2 error, largest row error, depth range
    and seconds per map (wall clock, profiler off)."""
    import torch
    from paper_2506_09551_gb300 import api, native

    native.load()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))

    def run(m, prec, stol, ctol, w_in, w):
        p = api.map_params(Gamma=0.3, eta=0.1, solve_tol=stol, cf_tol=ctol, precision=prec, cf_maxdepth=8000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        I, info, st = api.rixs_map(m, p, w_in, w)
        torch.cuda.synchronize()
        return I, {"seconds": time.perf_counter() - t0, "depth_min": info["cf_depth_min"],
                   "depth_max": info["cf_depth_max"]}

    def err(I, ref):
        rows = np.linalg.norm(I - ref, axis=1) / np.linalg.norm(ref, axis=1)
        return {"rel_l2": float(np.linalg.norm(I - ref) / np.linalg.norm(ref)), "row_max": float(rows.max())}

    out = []
    cases = [(workloads.CHAIN12, None, 1e-13, [(0, 1e-10, t) for t in (1e-11, 1e-10, 1e-9, 1e-8, 1e-7, 1e-6)] +
              [(1, 1e-8, t) for t in (1e-8, 1e-7, 1e-6, 1e-5, 1e-4)]),
             (workloads.CHAIN14, 10, 1e-11, [(1, 1e-8, t) for t in (1e-8, 1e-7, 1e-6, 1e-5, 1e-4)])]
    for wl, stride, ref_tol, runs in cases:
        m = api.model(wl.L, wl.n_up, wl.n_dn)
        w_in = wl.w_in[::stride] if stride else wl.w_in
        ref, r0 = run(m, 0, 1e-10, ref_tol, w_in, wl.w)
        out.append({"workload": wl.name, "n_w_in": len(w_in), "precision": "FP64", "cf_tol": ref_tol,
                    "reference": True, **r0})
        for prec, stol, ctol in runs:
            I, r = run(m, prec, stol, ctol, w_in, wl.w)
            rec = {"workload": wl.name, "n_w_in": len(w_in), "precision": "FP64" if prec == 0 else "FP32-mixed",
                   "solve_tol": stol, "cf_tol": ctol, **r, **err(I, ref)}
            out.append(rec)
            print(f"[bench] cf study {rec}", file=sys.stderr, flush=True)
    return {"metric": "continued-fraction stopping rule vs map error", "n_gpus": 1,
            "config": {"workload": args.workload}, "data": "synthetic", "study": out}


def gpu_arm(args, rank, world):
    import torch
    from paper_2506_09551_gb300 import api, native

    native.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    clusters = None
    if args.workload in CLUSTERS:
        clusters, prec, stol, ctol = CLUSTERS[args.workload]
        wl = clusters[-1]
        models = [api.model(c.L, c.n_up, c.n_dn, c.t, c.U, c.Uc, core_site=rank_core_site(rank, c.L))
                  for c in clusters]
    else:
        wl, prec, stol, ctol = WORKLOADS[args.workload]
    core = rank_core_site(rank, wl.L)
    m = api.model(wl.L, wl.n_up, wl.n_dn, wl.t, wl.U, wl.Uc, core_site=core)
    p = api.map_params(Gamma=wl.Gamma, eta=wl.eta, gs_tol=wl.gs_tol, solve_tol=stol, cf_tol=ctol, precision=prec)
    H = api.Operator.hubbard(m, False)
    Hp = api.Operator.hubbard(m, True)
    w_in, w = wl.w_in, wl.w
    if args.n_in:
        w_in = np.linspace(wl.w_in_range[0], wl.w_in_range[1], args.n_in)
    out = torch.empty((len(w_in), len(w)), dtype=torch.float64, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    lib = native.load()
    sites = SITES.get(args.workload)

    n_q = QMAPS.get(args.workload, 0)
    qs = 2 * np.pi * np.arange(n_q) / wl.L if n_q else None

    def one_map():
        if n_q:
            return api.rixs_map_q(m, p, qs, w_in, w)
        if clusters:
            I, E, info, st = api.rixs_map_clusters(models, p, w_in, w)
            return I, info, st
        if sites:
            return api.rixs_map_sites(m, p, sites, w_in, w)
        return api.rixs_map_ops(H, Hp, p, w_in, w, out=out)

    # launch choices measured on this GPU before the warm-up (untimed): the lag of the
    # per-shift update and the shape of the continued-fraction apply, cached by the
    # library for the maps below
    tuned = None
    if not args.no_autotune and not (n_q or clusters or sites):
        t_at = time.perf_counter()
        tuned = api.autotune(m, prec, len(w_in))
        tuned["seconds"] = time.perf_counter() - t_at
        print(f"[bench] autotune: {tuned}", file=sys.stderr, flush=True)
    for _ in range(args.warmup):
        one_map()
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    gpu_id = str(local)
    try:
        u = torch.cuda.get_device_properties(local).uuid
        gpu_id = "GPU-" + str(u) if not str(u).startswith("GPU-") else str(u)
    except Exception:
        pass
    # The timed steps run the product path (profiler off: the solve replays its CUDA graphs).
    with ClockSampler(None if args.no_clocks else gpu_id) as clk:
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            _, info, st = one_map()
            infos.append(info)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.summary()
    ms = max_over_ranks(ms, world)          # whole-job time = the slowest rank's
    n_maps = len(clusters) if clusters else (len(sites) if sites else (n_q or 1))
    pts = len(w_in) * len(w) * n_maps
    value = job_throughput(pts, world, ms * 1e-3)
    I_timed = out.cpu().numpy() if not (sites or clusters or n_q) else None
    print(f"[bench] {args.workload}: {ms:.1f} ms per map over {args.steps} steps", file=sys.stderr, flush=True)

    # One more step with the library profiler on: every launch bracketed by CUDA events on
    # its stream, for the kernel shares and the dominant kernel's roofline.
    torch.cuda.synchronize()
    lib.msb_profile_reset()
    lib.msb_profile_enable(1)
    one_map()
    torch.cuda.synchronize()
    lib.msb_profile_enable(0)
    stats = native.profile_read()

    # end to end through the public host API (operators built, grids in, map out)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    I_host = None
    if args.no_e2e:
        pass
    elif sites or clusters or n_q:
        one_map()          # already the host API: grids in from the host, maps out to the host
    else:
        I_host, info_e2e, _ = api.rixs_map(m, p, w_in, w)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    same = (float(np.max(np.abs(I_timed - I_host)) / np.max(np.abs(I_host)))
            if I_host is not None and np.max(np.abs(I_host)) > 0 else None)

    # The precision comparison: the same map once in the plain FP64 form on the same GPU.
    precision_cmp = None
    if args.workload in FP64_FORM and not args.no_fp64_leg:
        _, prec64, stol64, ctol64 = WORKLOADS[FP64_FORM[args.workload]]
        p64 = api.map_params(Gamma=wl.Gamma, eta=wl.eta, gs_tol=wl.gs_tol, solve_tol=stol64, cf_tol=ctol64,
                             precision=prec64)
        out64 = torch.empty_like(out)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        _, info64, st64 = api.rixs_map_ops(H, Hp, p64, w_in, w, out=out64)
        f1.record(stream)
        f1.synchronize()
        s64 = f0.elapsed_time(f1) * 1e-3
        I64 = out64.cpu().numpy()
        del out64
        precision_cmp = {
            "fp64_workload": FP64_FORM[args.workload], "fp64_seconds": s64,
            "fp64_value": len(w_in) * len(w) / s64, "mixed_seconds": ms * 1e-3,
            "fp32_vs_fp64_speedup": s64 / (ms * 1e-3),
            "rel_l2_mixed_vs_fp64": float(np.linalg.norm(I_timed - I64) / np.linalg.norm(I64)),
            "fp64_solve_tol": stol64, "fp64_cf_tol": ctol64, "fp64_n_w_in": len(w_in),
            "fp64_cf_depth_min": info64["cf_depth_min"], "fp64_cf_depth_max": info64["cf_depth_max"],
            "what": "one FP64 map of the same model and grid (profiler off, CUDA events), against the "
                    "timed FP32-mixed maps; the relative L2 difference of the two maps"}
        print(f"[bench] FP64 form: {s64:.2f} s per map, speed-up {s64 / (ms * 1e-3):.2f}x, "
              f"map difference {precision_cmp['rel_l2_mixed_vs_fp64']:.2e}", file=sys.stderr, flush=True)

    peaks = measured_peaks()
    # the continued-fraction apply shape that ran: the autotuned one, else the default
    # (FP32 shape 1; FP64 128 threads for rows up to 1024, else 256)
    ddn = math.comb(wl.L, wl.n_dn)
    shape = tuned["cf_threads"] if tuned and tuned.get("cf_threads") else (1 if prec else (128 if ddn <= 1024 else 256))
    top, roof = dominant_roofline(stats, prec, peaks, args.workload, shape)
    total_ms = sum(s["ms"] for s in stats)
    apply_cls = [s for s in stats if s["name"] in ("cf_apply", "seed_mvm", "h_apply")]
    h_gbs = (sum(s["alg_bytes"] for s in apply_cls) / (sum(s["ms"] for s in apply_cls) * 1e-3) / 1e9
             if apply_cls else None)
    launches = int(sum(i["kernel_launches"] for i in infos) / args.steps)
    line = {
        "metric": "RIXS map (w_in, w) points/s",
        "value": value,
        "unit": "map points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c128" if prec == 0 else "c64 vectors, f64 scalars",
        "data": "synthetic: 1D Hubbard ring, random-start Lanczos ground state",
        "config": {"workload": args.workload, "L": wl.L, "n_up": wl.n_up, "n_dn": wl.n_dn,
                   "dim_ground": int(H.dim), "dim_intermediate": int(Hp.dim), "n_w_in": len(w_in), "n_w": len(w),
                   "Gamma": wl.Gamma, "eta": wl.eta, "solve_tol": stol, "cf_tol": ctol,
                   "precision": "FP64" if prec == 0 else "FP32-mixed",
                   "parallelism": f"{world} independent maps (core site = rank)",
                   "l2": "working set (vectors of GBs) larger than L2; no flush needed"},
        "e2e": None if args.no_e2e else {
            "value": job_throughput(pts, world, e2e_s), "unit": "map points/s",
            "h2d_bytes_per_step": int(8 * (len(w_in) + len(w))) + 2 * 8 * 4,
            "d2h_bytes_per_step": int(8 * pts), "seconds": e2e_s,
            "max_rel_diff_vs_value_map": same},
        "gpu_launches": launches,
        "roofline": roof,
        "h_apply_alg_gbs": h_gbs,
        "clocks": clocks,
        "precision_comparison": precision_cmp,
        "autotune": tuned,
        "profiled_step": "kernel shares and roofline from one extra map with the library profiler on",
        "solve": {k: infos[-1][k] for k in ("iterations", "n_converged", "matvecs", "cf_depth_max",
                                            "cf_depth_min", "seconds_ground_state", "seconds_solve",
                                            "seconds_second_step", "device_bytes", "E_G")},
        "kernels": sorted([{"name": s["name"], "launches": s["launches"], "ms": round(s["ms"], 3),
                            "share": round(s["ms"] / total_ms, 4)} for s in stats],
                          key=lambda d: -d["ms"]),
    }
    if clusters:
        # batched vs the same clusters as separate calls, both by wall clock with the
        # library profiler off (one pass each)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_map()
        torch.cuda.synchronize()
        t_batched = time.perf_counter() - t0
        t0 = time.perf_counter()
        for mc in models:
            api.rixs_map(mc, p, w_in, w)
        torch.cuda.synchronize()
        line["separate_maps"] = {"separate_seconds": time.perf_counter() - t0, "batched_seconds": t_batched,
                                 "what": "wall clock, profiler off: one msb_rixs_map_clusters call vs one "
                                         "msb_rixs_map call per cluster"}
        line["config"]["clusters"] = [
            {"L": c.L, "n_up": c.n_up, "n_dn": c.n_dn, "dim_ground": math.comb(c.L, c.n_up) * math.comb(c.L, c.n_dn),
             "dim_intermediate": math.comb(c.L, c.n_up + 1) * math.comb(c.L, c.n_dn)} for c in clusters]
        line["config"]["parallelism"] = (f"{world} x (one solve on the direct sum of the clusters' H', "
                                         "one continued fraction over all their columns)")
        for k in ("L", "n_up", "n_dn", "dim_ground", "dim_intermediate"):
            line["config"].pop(k)
    return line


def reference_arm(args) -> dict:
    """The oracle on the host cores, for the same workload, metric and unit: each step is
    the cpu_baseline measurement of that workload (the whole map for small workloads,
    the bounded all-core sample scaled to a whole map for large ones)."""
    if args.workload not in WORKLOADS:
        return {"impl": "reference",
                "unavailable": f"the oracle baseline covers the single-map Hubbard workloads, not {args.workload}"}
    wl = WORKLOADS[args.workload][0]
    vals = []
    for i in range(args.warmup + args.steps):
        r = run_cpu_baseline(args.workload)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.mean([r["value"] for r in vals if r["value"]]) if any(r["value"] for r in vals) else None
    ms = wl.n_in * wl.n_w / v * 1e3 if v else None
    cb = dict(vals[-1])
    cb["value"] = v
    return {"metric": "RIXS map (w_in, w) points/s", "value": v, "unit": "map points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "impl": "reference", "config": {"workload": args.workload},
            "estimate": bool(cb.get("estimate", False)),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "map points/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(CSR_WORKLOADS) + sorted(CLUSTERS) + [SWEEP, CF_STUDY],
                    default=DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end map (profiling runs)")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi (profiling runs)")
    ap.add_argument("--n-in", type=int, default=0, help="incident energies (0: the workload's; profiling runs)")
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64 form of an FP32-mixed workload")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch choices (no trials before the warm-up)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload in (SWEEP, CF_STUDY):
        if rank == 0:
            fn = gpu_arm_sweep if args.workload == SWEEP else gpu_arm_cf_study
            print(json.dumps(fn(args, rank, world)), flush=True)
        return
    if args.workload in CSR_WORKLOADS:
        line = gpu_arm_csr(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    line = gpu_arm(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = run_cpu_baseline(args.workload)
            if args.workload == DEFAULT:
                try:
                    line["cpu_full_small_map"] = cpu_full_map(workloads.CHAIN8)
                except Exception as e:
                    line["cpu_full_small_map"] = {"value": None, "sample": f"failed: {type(e).__name__}: {e}"}
        elif not args.no_cpu_baseline:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
