#!/usr/bin/env python
"""Benchmark: RIXS map throughput (incident x loss energy points per second).

One step = one whole RIXS map of the workload (Eqs. 1-2): Hubbard operators,
FP64 Lanczos ground state, the multi-shifted BiCG solve for every incident
energy, the sector maps and the batched continued fraction of the second step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` times msb_rixs_map_ops (operators
built beforehand, map left on the device) with CUDA events on the calling
stream; `e2e` times msb_rixs_map (host grids in, host map out, operators
built inside the call) with a wall clock.  Every kernel launch inside the
timed steps is bracketed by CUDA events by the library's profiler, which
gives the dominant kernel's achieved bandwidth / FLOP rate for `roofline`.
Under torchrun each rank computes the map of its own core site (independent
problems, no collective on the data path): weak scaling.

Workloads (--workload): hubbard-L12-fp64 (default), hubbard-L8-fp64,
hubbard-L14-mixed, hubbard-L14-fp64 (the same ring in FP64, for the precision
comparison; use --n-in to shorten it), hubbard-L12x12rhs-mixed (one right-hand
side per core site, one call), hubbard-L10-11-12-clusters-mixed (three clusters
of uneven size in one solve and one continued fraction; its line adds
`separate_maps`, the same clusters as separate calls), hubbard-L12-q12-mixed
(momentum-resolved maps: the coherent sum over the 12 core sites at the 12
momenta 2 pi k / 12), random-csr-fp64 and
random-csr-mixed (n = 2^22, 256 shifts; one step = the multi-shift solve).
`cpu_baseline` (the oracle on one host core, a bounded sample scaled to the
whole map) is sampled for the single-map workloads up to L = 12.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

# name -> (workload, precision, solve_tol, cf_tol)
WORKLOADS = {
    "hubbard-L12-fp64": (workloads.CHAIN12, 0, 1e-10, 1e-10),
    "hubbard-L14-mixed": (workloads.CHAIN14, 1, 1e-8, 1e-8),
    "hubbard-L14-fp64": (workloads.CHAIN14, 0, 1e-10, 1e-10),
    "hubbard-L8-fp64": (workloads.CHAIN8, 0, 1e-10, 1e-10),
    "hubbard-L12x12rhs-mixed": (workloads.BATCH_SITES, 1, 1e-8, 1e-8),
    "hubbard-L12-q12-mixed": (workloads.BATCH_SITES, 1, 1e-8, 1e-8),
}
# workloads with one right-hand side per core site (one call, one shared second step)
SITES = {"hubbard-L12x12rhs-mixed": list(range(12))}
# momentum-resolved maps (coherent sum over all core sites): name -> number of momenta 2 pi k / L
QMAPS = {"hubbard-L12-q12-mixed": 12}
# clusters of uneven size in one call: name -> (clusters, precision, solve_tol, cf_tol)
CLUSTERS = {"hubbard-L10-11-12-clusters-mixed": (workloads.BATCH_CLUSTERS, 1, 1e-8, 1e-8)}
DEFAULT = "hubbard-L12-fp64"
# random complex-symmetric stress workload: name -> precision, tolerance
CSR_WORKLOADS = {"random-csr-fp64": (0, 1e-10), "random-csr-mixed": (1, 1e-7)}

# Roofline denominators.  HBM: the measured copy bandwidth of this machine.  FP64:
# 152 SMs x 2 FP64 FMA per clock x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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
# CPU baseline: the oracle, single-threaded, on a bounded sample
# ---------------------------------------------------------------------------
def oracle_costs(name: str):
    path = os.path.join(ROOT, "profiles", f"oracle_costs_{name}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def cpu_baseline_worker(name: str, n_iter: int = 20) -> dict:
    """Runs in a fresh single-threaded process: build, ground state, and a
    bounded number of BiCGStab iterations / continued-fraction steps of one
    row of the map, all with the oracle's own functions.  The whole map's time
    is scaled from these with the oracle's per-row counts for this workload."""
    import scipy.sparse as sp
    from oracle import hubbard, solvers, spectrum
    wl = WORKLOADS[name][0]
    t0 = time.perf_counter()
    m = hubbard.RixsModel(wl.L, wl.n_up, wl.n_dn, wl.t, wl.U, wl.Uc, wl.core_site)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    E_G, G, _ = solvers.ground_state(m.H, workloads.lanczos_start(m.H.shape[0], wl.lanczos_seed), kmax=300)
    t_gs = time.perf_counter() - t0
    k = wl.n_in // 2
    n = m.Hp.shape[0]
    A = (m.Hp - (E_G + wl.w_in[k] + 1j * wl.Gamma) * sp.identity(n)).tocsr()
    b = (m.O2 @ G).astype(np.complex128)
    t0 = time.perf_counter()
    x, nmv = solvers.bicgstab(lambda v: A @ v, b, 1e-13, maxit=n_iter, restarts=1, strict=False)
    t_solve = time.perf_counter() - t0
    lz = spectrum._Lanczos(m.H, m.O1 @ x)
    t0 = time.perf_counter()
    lz.advance(n_iter)
    t_cf = time.perf_counter() - t0
    costs = oracle_costs(name)
    per_mv = t_solve / max(nmv, 1)
    per_step = t_cf / max(len(lz.a), 1)
    if costs:
        mv_row, depth_row = costs["mean_solve_matvecs"], costs["mean_cf_depth"]
        src = f"per-row counts from profiles/oracle_costs_{name}.json ({len(costs['rows'])} rows run in full)"
    else:
        mv_row, depth_row = float("nan"), float("nan")
        src = "no recorded per-row counts"
    T_map = t_build + t_gs + wl.n_in * (mv_row * per_mv + depth_row * per_step)
    pts = wl.n_in * wl.n_w
    return {
        "value": pts / T_map, "unit": "map points/s", "cores": 1, "kind": "oracle",
        "sample": (f"oracle (numpy/scipy, 1 thread) on {name}: build H,H' ({t_build:.1f}s), Lanczos ground state "
                   f"({t_gs:.1f}s), {nmv} BiCGStab MVMs and {len(lz.a)} CF Lanczos steps of row {k} "
                   f"({t_solve + t_cf:.1f}s); whole map = build + ground state + {wl.n_in} rows x "
                   f"({mv_row:.0f} MVMs + {depth_row:.0f} CF steps), {src}"),
        "seconds_measured": t_build + t_gs + t_solve + t_cf,
        "map_seconds_scaled": T_map,
    }


# The oracle builds H and H' in CSR and runs a ground-state Lanczos of up to 300
# steps with full reorthogonalisation: bounded samples are feasible up to L = 12
# (D < 10^6); at L = 14 the build and ground state alone run far beyond the bound.
ORACLE_MAX_DIM = 1_000_000


def oracle_feasible(name: str) -> bool:
    if name not in WORKLOADS:
        return False
    wl = WORKLOADS[name][0]
    return math.comb(wl.L, wl.n_up) * math.comb(wl.L, wl.n_dn) <= ORACLE_MAX_DIM


def run_cpu_baseline(name: str) -> dict:
    if not oracle_feasible(name):
        return {"value": None, "unit": "map points/s", "cores": 1, "kind": "oracle",
                "sample": f"not sampled: the oracle's build and ground state at {name} exceed the bounded sample"}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", "--workload", name],
                       capture_output=True, text=True, env=env, timeout=900)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    return {"value": None, "unit": "map points/s", "cores": 1, "kind": "oracle",
            "sample": "failed: " + (r.stderr.strip().splitlines() or ["?"])[-1]}


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
def measured_traffic(workload, kernel, alg_bytes_per_launch):
    """DRAM bytes per launch scaled from an ncu capture of the same kernel (None if none)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[workload][kernel]
    except (OSError, KeyError, ValueError):
        return None
    return rec["dram_bytes"] / rec["alg_bytes"] * alg_bytes_per_launch


def dominant_roofline(stats, prec, peaks, workload=None):
    top = max(stats, key=lambda s: s["ms"])
    avg_ms = top["ms"] / top["launches"]
    traffic = measured_traffic(workload, top["name"], top["alg_bytes"] / top["launches"])
    if prec == 0 and top["name"] != "cf_apply":
        # FP64 complex multiply-adds per shift (the per-shift update): FP64-pipe bound
        achieved = top["alg_flops"] / top["launches"] / (avg_ms * 1e-3) / 1e12
        return top, {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": top["name"],
                     "peak_source": "derived FP64: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz"}
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

    for _ in range(args.warmup):
        x, per, info, st = step()
        del x
    torch.cuda.synchronize()
    barrier()
    lib.msb_profile_reset()
    lib.msb_profile_enable(1)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None if args.no_clocks else str(local)) as clk:
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            x, per, info, st = step()
        e1.record(stream)
        e1.synchronize()
    lib.msb_profile_enable(0)
    stats = native.profile_read()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
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
        "solve": {"iterations": info["iterations"], "n_converged": info["n_converged"],
                  "max_shift_residual": info["max_shift_residual"], "device_bytes": info["device_bytes"]},
        "kernels": sorted([{"name": s_["name"], "launches": s_["launches"], "ms": round(s_["ms"], 3),
                            "share": round(s_["ms"] / total_ms, 4)} for s_ in stats], key=lambda d: -d["ms"]),
        "cpu_baseline": None,
    }


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

    for _ in range(args.warmup):
        one_map()
    torch.cuda.synchronize()
    barrier()
    lib.msb_profile_reset()
    lib.msb_profile_enable(1)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    gpu_id = str(local)
    try:
        u = torch.cuda.get_device_properties(local).uuid
        gpu_id = "GPU-" + str(u) if not str(u).startswith("GPU-") else str(u)
    except Exception:
        pass
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
    lib.msb_profile_enable(0)
    stats = native.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.summary()
    ms = max_over_ranks(ms, world)          # whole-job time = the slowest rank's
    n_maps = len(clusters) if clusters else (len(sites) if sites else (n_q or 1))
    pts = len(w_in) * len(w) * n_maps
    value = job_throughput(pts, world, ms * 1e-3)

    print(f"[bench] {args.workload}: {ms:.1f} ms per map over {args.steps} steps", file=sys.stderr, flush=True)
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
    I_dev = out.cpu().numpy()
    same = (float(np.max(np.abs(I_dev - I_host)) / np.max(np.abs(I_host)))
            if I_host is not None and np.max(np.abs(I_host)) > 0 else None)

    peaks = measured_peaks()
    top, roof = dominant_roofline(stats, prec, peaks, args.workload)
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
    """The oracle on the host cores: each step is a bounded sample of the same
    workload (see cpu_baseline_worker), scaled to a whole map."""
    if not oracle_feasible(args.workload):
        return {"impl": "reference",
                "unavailable": f"the oracle's bounded sample covers the single-map workloads up to L = 12, "
                               f"not {args.workload}"}
    wl, prec, stol, ctol = WORKLOADS[args.workload]
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
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "map points/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(CSR_WORKLOADS) + sorted(CLUSTERS),
                    default=DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end map (profiling runs)")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi (profiling runs)")
    ap.add_argument("--n-in", type=int, default=0, help="incident energies (0: the workload's; profiling runs)")
    ap.add_argument("--cpu-baseline-worker", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.cpu_baseline_worker:
        print(json.dumps(cpu_baseline_worker(args.workload)))
        return

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
        elif not args.no_cpu_baseline:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
