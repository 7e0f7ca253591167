"""Benchmark: K-Means solves/s to convergence, Anderson-accelerated vs plain Lloyd, on one GB300.

Default workload ``dense_1m`` (the largest single-GPU configuration): N = 1,000,000, d = 128,
K = 1024, X in BF16 with the FP32 copy, 1024 full-covariance Gaussians, distances on the tcgen05
tensor cores.  ``--workload lowd_2m``: N = 2,000,000 samples, d = 3, K = 256, FP32, a mixture of
256 anisotropic Gaussians (axis std log-U[0.1, 2], centres U[0,100]^3, Dirichlet(1) weights).
One data set (seed 0); each step starts from its own C0 (K distinct samples, seed 1000 + step).
A step is one full solve to convergence (tol = 0, max_iter = 1000) through the C ABI with X
resident in HBM; L2 is flushed (256 MB write) before every step, outside the step's CUDA events.

Prints one JSON line.  The CPU leg (skipped with --no-cpu-baseline) runs the FP64 oracle on the
host cores: the baseline timing on the full-size problem, and the error of the first solves'
results against FP64 arithmetic.  ``--impl reference`` times the same oracle as the reference arm.
Multi-GPU (torchrun): independent replicas per rank (no data-path collective), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import datagen  # noqa: E402

METRIC = "K-Means solves/s to convergence, AA vs plain Lloyd, same GB300; p50/p99 latency"
WORKLOADS = {
    "lowd_2m": dict(workload="lowd_2m", N=2_000_000, d=3, K=256, m_max=10, data_seed=0,
                    init="K distinct samples, seed 1000+step", dtype="f32"),
    "dense_1m": dict(workload="dense_1m", N=1_000_000, d=128, K=1024, m_max=10, data_seed=0,
                     init="K distinct samples, seed 1000+step", dtype="bf16 distances, f32 X"),
}
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def calibrated_fp32_peak():
    """Measured FP32 FMA rate (T lane-op/s) from the committed calibration summary, or None."""
    try:
        for ln in open(os.path.join(ROOT, "profiles", "fp32_fma_peak.md")):
            if ln.startswith("| measured FP32 FMA peak"):
                return float(ln.split("|")[2].split()[0])
    except (OSError, ValueError, IndexError):
        return None
    return None


def profiled_traffic(name: str):
    """DRAM bytes per launch (read + write) of the dominant kernel from its committed ncu summary."""
    try:
        for ln in open(os.path.join(ROOT, "profiles", name)):
            if ln.startswith("| traffic per launch"):
                return int(ln.split("|")[2].split()[0])
    except (OSError, ValueError, IndexError):
        return None
    return None


def dense_inc() -> bool:
    """The dense solver passes' incremental update (KM_DINC=0 switches it off)."""
    return not os.environ.get("KM_DINC", "1").startswith("0")


def solve_launches(iters: int, dense: bool, ham: bool, fused_mix: bool, rejected: int = 0,
                   inc: bool = True) -> int:
    """Kernels one solve launches.  Low-d: the prologue (k_prep, [k_hprep], INIT pass, k_fin,
    [k_mix]), per loop pass the same with the TRIAL and REVERT passes in place of the INIT pass,
    and the epilogue (EPI pass, k_epi); k_hprep with Hamerly bounds, k_mix unless the mix is fused
    into k_fin.  Dense (with its Hamerly bounds): 14 in the prologue (k_prep, k_xcheck, two
    packings, the INIT chain of 8: drifts, assignment, rescan, rescan labels, count, scan, scatter,
    segment sums; k_fin, k_mix), per loop pass 13 (the TRIAL chain of 10: drifts, bounds test, row
    gather and the 7 of the INIT chain; k_fin, k_mix, the packing) plus the REVERT chain's 10 when
    the safeguard fired (it sits in a conditional node otherwise), 5 in the epilogue.  The
    incremental update adds three kernels to every INIT, TRIAL and REVERT chain (the changed-row
    list, their sums, the new sums with the energy)."""
    if dense:
        k = 3 if inc else 0
        return 19 + k + (13 + k) * iters + (10 + k) * rejected
    per = 3 + int(ham) + int(not fused_mix)
    return per * (iters + 1) + 2


def batched_launches(loops: int, ngrp: int, ham: bool, mix: bool, dense_iters) -> int:
    # dense_iters: (iterations, rejected) of each tensor-core instance
    """Kernels of one batched solve.  Low-d chain: prologue (k_prep_batch, [k_hprep_batch], one
    INIT pass per group, k_fin_batch, [k_mix_batch]), per loop step ([k_hprep_batch], TRIAL and
    REVERT passes per group, k_fin_batch, [k_mix_batch], k_batch_done), epilogue (EPI pass per
    group, k_epi_batch); plus one tensor-core chain per dense instance."""
    h, m = int(ham), int(mix)
    lowd = (2 + h + ngrp + m) + loops * (h + 2 * ngrp + 2 + m) + ngrp + 1 if ngrp else 0
    return lowd + sum(solve_launches(it, True, False, False, rj, dense_inc()) for it, rj in dense_iters)


def same_energy_speed(ms_aa, ms_ll, E_aa, E_ll, rtol: float = 1e-6):
    """Lloyd's time over Algorithm 1's on the initialisations where both end at the same energy
    (within rtol), and how many there were; (None, 0) when there are none."""
    same = [i for i in range(len(ms_aa)) if abs(E_aa[i] - E_ll[i]) <= rtol * abs(E_ll[i])]
    if not same:
        return None, 0
    return sum(ms_ll[i] for i in same) / sum(ms_aa[i] for i in same), len(same)


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest replica sets the job time); `dist`
    is torch.distributed or None for a single process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    i = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[i]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def load_data(wl, rows=0):
    """(X f32, X_bf16 uint16 or None) of the workload (rows > 0: that many rows of the same
    generator, a smaller case for profiler captures)."""
    kw = dict(N=rows) if rows > 0 else {}
    if wl["workload"] == "dense_1m":
        X, Xb, _ = datagen.dense_1m(seed=wl["data_seed"], **kw)
        return X, Xb
    X, _ = datagen.lowd_2m(seed=wl["data_seed"], **kw)
    return X, None


# ----------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            self.path = os.path.join(tempfile.gettempdir(), f"km_clocks_{os.getpid()}.csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ CPU oracle
def oracle_timed(X, C0, max_iter: int, m_max: int, lloyd: bool = False, threads: int = 0):
    """One FP64 oracle solve of the full-size problem, capped at max_iter loop passes; returns
    (seconds, info, cores).  threads > 0 runs it on that many threads (then back)."""
    import oracle
    prev = oracle.num_threads()
    if threads > 0:
        oracle.set_num_threads(threads)
    try:
        t0 = time.perf_counter()
        C, rho, info = oracle.solve(X, C0, lloyd=lloyd, m_max=m_max, max_iter=max_iter)
        return time.perf_counter() - t0, info, oracle.num_threads(), C, rho
    finally:
        oracle.set_num_threads(prev)


def oracle_dense_passes(path=None):
    """Assignment passes of the FP64 oracle's full-size Algorithm 1 solve on dense_1m from the
    first step's C0 (written by tests/golden/make_dense_1m.py, which calls only the oracle)."""
    path = path or os.path.join(ROOT, "tests", "golden", "dense_1m_oracle.json")
    try:
        return int(json.load(open(path))["aa"]["assign_passes"])
    except (OSError, ValueError, KeyError):
        return None


def result_errors(X, results, sample_rows: int = 4000):
    """Error of returned results against FP64 arithmetic on the same assignment (the oracle):
    per result (C, rho, E) the relative energy error |E - E(P, C)| / E(P, C), the relative
    centroid error ||C - means(P)|| / ||means(P)|| (Eq. 4 in FP64), and, on a row sample, labels
    that differ from the FP64 argmin at C on rows whose top-2 gap is clear of 1e-6 * max(||x||^2,
    ||c||^2) (must be 0) and rows inside that band (either label is correct to the tolerance)."""
    import oracle
    r = np.random.default_rng(2024)
    idx = np.sort(r.choice(X.shape[0], size=min(sample_rows, X.shape[0]), replace=False))
    Xs = X[idx].astype(np.float64)
    eE, eC, bad, band = [], [], 0, 0
    for C, rho, E in results:
        C64 = C.astype(np.float64)
        E_o = oracle.energy(X, C64, rho)
        G_o, _ = oracle.update(X, rho, C.shape[0], C64)
        eE.append(abs(E - E_o) / E_o)
        eC.append(float(np.linalg.norm(C64 - G_o) / np.linalg.norm(G_o)))
        ro, dmin, gap = oracle.assign(Xs, C64)
        xn = (Xs * Xs).sum(1)
        cn = (C64 * C64).sum(1)
        clear = gap > 1e-6 * np.maximum(xn, cn.max())
        bad += int(((rho[idx] != ro) & clear).sum())
        band += int((~clear).sum())
    return {"E_rel_max": max(eE), "C_rel_max": max(eC), "solves": len(results), "rows_sampled": len(idx),
            "labels_off_argmin_clear_rows": bad, "rows_in_tie_band": band,
            "what": "returned (C, P, E) against FP64 oracle arithmetic: E(P, C) of Eq. 1, the means of P "
                    "(Eq. 4), the FP64 argmin (Eq. 3) at C on a row sample"}


def reference_sample(args):
    """Oracle (FP64, host cores) over a bounded sample of the batched or serving workload:
    (instance solves/s, cores, description of the sample)."""
    import oracle
    if args.workload == "batched_512":
        shapes = [sh for sh in datagen.batched_shapes(args.batch_instances, seed=0) if sh[1] <= 16 and sh[0] <= 20000]
        what = "low-d batched_512 instances with N <= 20000"
    else:
        reqs = datagen.serving_stream(args.serve_requests, rate=args.serve_rate, seed=7)
        shapes = [(q["N"], q["d"], q["K"], q["data_seed"]) for q in reqs[::100] if not q["large"] and q["d"] <= 16]
        what = "every 100th serving request with d <= 16"
    shapes = shapes[:max(1, args.steps) * 4]
    t = 0.0
    for N, d, K, ds in shapes:
        X = datagen.isotropic_mixture(N, d, K, ds, dtype=np.float64)
        C0 = datagen.init_centroids(X, K, ds + 1000)
        t0 = time.perf_counter()
        oracle.solve(X, C0, m_max=10)
        t += time.perf_counter() - t0
    return len(shapes) / t, oracle.num_threads(), f"{len(shapes)} {what} (Algorithm 1, FP64)"


def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    if args.workload in ("batched_512", "serving"):
        value, cores, sample = reference_sample(args)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "instance solves/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload, "parallelism": "cpu-oracle"},
                "cpu_baseline": {"value": value, "unit": "instance solves/s", "cores": cores, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "instance solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    wl = WORKLOADS[args.workload]
    X, _ = load_data(wl)
    K = wl["K"]
    nsteps = max(1, min(args.steps, 3))
    C0s = [datagen.init_centroids(X, K, 1000 + s) for s in range(nsteps)]
    oracle_timed(X[:20_000], C0s[0][:min(K, 64)], 1, wl["m_max"])       # warm the thread pool
    if wl["d"] <= 16:
        # full-size solves to convergence, one per step
        times, infos = [], []
        for s in range(nsteps):
            t, info, cores, _, _ = oracle_timed(X, C0s[s], 1000, wl["m_max"])
            times.append(t)
            infos.append(info)
        value = nsteps / sum(times)
        sample = (f"{nsteps} full-size Algorithm 1 solves (N={X.shape[0]}, FP64, all host cores) from the "
                  f"C0 of steps 0..{nsteps - 1}; iterations {[i['iters'] for i in infos]}")
        step_ms = [1e3 * t for t in times]
    else:
        # full-size passes: time per assignment pass x the assignment passes of the oracle's full solve
        P_full = oracle_dense_passes()
        if P_full is None:
            print(json.dumps({"impl": "reference", "unavailable": "tests/golden/dense_1m_oracle.json missing"}))
            return
        per_pass, step_ms = [], []
        for s in range(nsteps):
            t, info, cores, _, _ = oracle_timed(X, C0s[s], 1, wl["m_max"])
            per_pass.append(t / info["assign_passes"])
            step_ms.append(1e3 * t)
        value = 1.0 / (float(np.mean(per_pass)) * P_full)
        sample = (f"Algorithm 1 on the full {X.shape[0]} x {X.shape[1]} problem (FP64, all host cores) from the "
                  f"C0 of steps 0..{nsteps - 1}, each stopped after its first loop pass (2 assignment passes); "
                  f"solves/s = 1 / (mean time per assignment pass {np.mean(per_pass):.2f} s x {P_full} assignment "
                  f"passes of the oracle's full-size solve from step 0's C0, tests/golden/dense_1m_oracle.json)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": nsteps, "warmup": 1,
        "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(wl, parallelism="cpu-oracle"),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": f"{nsteps} steps of the requested {args.steps}: each step is full-size oracle work",
    }
    print(json.dumps(line), flush=True)


def cpu_leg(args, wl, X, C0s, inf_aa, res_aa, res_ll):
    """The oracle on the host cores (rank 0, N = 1): the CPU baseline on the full-size problem and
    the error of the first returned results against FP64 arithmetic."""
    m_max = wl["m_max"]
    C0 = C0s[args.warmup]
    gpu_passes = float(np.mean([i["assign_passes"] for i in inf_aa]))
    out = {}
    if wl["d"] <= 16:
        n = max(1, args.cpu_solves)
        times, infos, Es = [], [], []
        for s in range(n):
            t, info, cores, C, rho = oracle_timed(X, C0s[args.warmup + s], 1000, m_max)
            times.append(t)
            infos.append(info)
        base = {"value": n / sum(times), "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"{n} full-size Algorithm 1 solves (FP64) from the C0 of the first {n} timed steps"}
        # the same C0 on the GPU: a reduced-precision solve may take the other branch of a safeguard
        # comparison and stop at a neighbouring fixed point (its energy then differs slightly)
        out["vs_oracle_solve"] = [{"iters_gpu": r[3]["iters"], "iters_oracle": i["iters"],
                                   "rejected_gpu": r[3]["rejected"], "rejected_oracle": i["rejected"],
                                   "E_rel": abs(r[2] - i["E"]) / i["E"]} for r, i in zip(res_aa, infos)]
        t1, info1, _, _, _ = oracle_timed(X, C0, 1, m_max, threads=1)
        per1 = t1 / info1["assign_passes"]
        base["value_1_thread"] = 1.0 / (per1 * float(np.mean([i["assign_passes"] for i in infos])))
        base["sample_1_thread"] = ("one thread: time per assignment pass of a full-size solve stopped after its first "
                                   "loop pass x the assignment passes of the full solves above")
    else:
        t, info, cores, _, _ = oracle_timed(X, C0, 1, m_max)
        per = t / info["assign_passes"]
        P_full = oracle_dense_passes()
        base = {"value": 1.0 / (per * gpu_passes), "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"Algorithm 1 on the full {X.shape[0]} x {X.shape[1]} problem (FP64) from the first timed "
                          f"step's C0, stopped after its first loop pass ({info['assign_passes']} assignment passes, "
                          f"{t:.1f} s): time per assignment pass x the mean assignment passes of the timed solves "
                          f"({gpu_passes:.1f}); the oracle's own full solve from step 0's C0 takes {P_full}"}
        rows = 62_500
        t1, info1, _, _, _ = oracle_timed(X[:rows], C0, 1, m_max, threads=1)
        per1 = t1 / info1["assign_passes"] * (X.shape[0] / rows)
        base["value_1_thread"] = 1.0 / (per1 * gpu_passes)
        base["sample_1_thread"] = (f"one thread: time per assignment pass on the first {rows} rows x {X.shape[0] // rows} "
                                   "(a pass is linear in N) x the mean assignment passes of the timed solves")
    out["cpu_baseline"] = base
    out["err_vs_oracle"] = {"aa": result_errors(X, [(C, r, E) for C, r, E, _ in res_aa]),
                            "lloyd": result_errors(X, [(C, r, E) for C, r, E, _ in res_ll])}
    return out


# ------------------------------------------------------------------- batched and serving data
def batched_data(n_inst: int, seed: int = 0):
    """The uneven batched workload: per instance (X f32, X_bf16 bits or None, K, data_seed)."""
    out = []
    for N, d, K, ds in datagen.batched_shapes(n_inst, seed=seed):
        X = datagen.isotropic_mixture(N, d, K, ds, dtype=np.float32)
        out.append((X, datagen.to_bf16_bits(X) if d > 16 else None, K, ds))
    return out


def parse_tuning(desc: str):
    """Per low-d group of kmeans_batch_describe: (d, lane ops of one pass, chosen grid, its time in
    us).  A group reads "... v0(occ 3) 152:528.4us ... v1(occ 3) ... -> variant V grid G"."""
    out = []
    for part in desc.split(";"):
        part = part.strip()
        if " d=" not in part or "-> variant" not in part:
            continue
        d = int(part.split(" d=")[1].split()[0])
        ops = float(part.split(" ops=")[1].split()[0])
        tail = part.split("-> variant")[1].split()
        var, grid = int(tail[0]), int(tail[2])
        t = None
        cur = None
        for tok in part.split("->")[0].split():
            if tok.startswith("v") and "(occ" in tok:
                cur = int(tok[1:tok.index("(")])
            elif cur == var and tok.startswith(f"{grid}:") and tok.endswith("us"):
                t = float(tok[len(str(grid)) + 1:-2])
        out.append((d, ops, grid, t))
    return out


def run_batched(args, rank, world, local_rank):
    """512 uneven instances (d in {2,3,16,64}) per step through kmeans_solve_batched."""
    import torch
    import paper_1805_10638_gb300 as km

    torch.cuda.set_device(local_rank)
    data = batched_data(args.batch_instances, seed=0)
    n = len(data)
    nsteps = args.steps + args.warmup
    ctx = km.Context(local_rank)
    stream = torch.cuda.current_stream()
    Xs = [torch.from_numpy(X).cuda() for X, _, _, _ in data]
    Xbs = [torch.from_numpy(b.view(np.int16)).cuda().view(torch.bfloat16) if b is not None else None
           for _, b, _, _ in data]
    C0host = [[datagen.init_centroids(X, K, ds + 1000 + s) for (X, _, K, ds) in data] for s in range(nsteps)]
    C0buf = [torch.empty((K, X.shape[1]), dtype=torch.float32, device="cuda") for X, _, K, _ in data]
    C0dev = [[torch.from_numpy(c).cuda() for c in row] for row in C0host]
    Couts = [torch.empty_like(c) for c in C0buf]
    rhos = [torch.empty(X.shape[0], dtype=torch.int32, device="cuda") for X, _, _, _ in data]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def load_c0(s):
        for i in range(n):
            C0buf[i].copy_(C0dev[s][i])

    def leg(lloyd: bool):
        prm = dict(max_iter=args.max_iter, **(dict(lloyd_only=1) if lloyd else dict(m_max=10)))
        for s in range(args.warmup):
            load_c0(s)
            km.kmeans_solve_batched(ctx, Xs, C0buf, Couts, rhos, params=prm, X_bf16s=Xbs)
        torch.cuda.synchronize()
        ms, infos = [], []
        for s in range(args.steps):
            flush.fill_(float(s))
            load_c0(args.warmup + s)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, inf, _ = km.kmeans_solve_batched(ctx, Xs, C0buf, Couts, rhos, params=prm, X_bf16s=Xbs)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(inf)
        return ms, infos, km.batch_describe(ctx)

    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_aa, inf_aa, desc = leg(False)
    ms_ll, inf_ll, _ = leg(True)
    clk = clocks.stop()
    tot_aa, tot_ll = sum(ms_aa) / 1e3, sum(ms_ll) / 1e3

    # roofline of the batched low-d assignment pass: the tuner's timing of the chosen grid per group
    groups = parse_tuning(desc)
    work, t_us = 0.0, 0.0
    for d, ops, grid, t in groups:
        if t is None:
            continue
        work += ops
        t_us += t
    peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2070.0 * 1e6 / 1e12
    achieved = work / (t_us * 1e-6) / 1e12 if t_us else None
    roof = {"bound": "alu", "kernel": "k_pass_lowd_batch (all low-d instances, one pass per group)",
            "unit": "Tlane-op/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak if achieved else None, "traffic": None,
            "note": "sum over low-d instances of N*K*(d+2) lane ops over the summed per-group pass times the "
                    "autotuner measured for the grids it chose (CUDA events); peak as for lowd_2m"}

    # end to end: inputs from pinned host memory, results back to the host, through the public API
    Xh = [torch.from_numpy(X).pin_memory() for X, _, _, _ in data]
    Xbh = [torch.from_numpy(b.view(np.int16)).pin_memory() if b is not None else None for _, b, _, _ in data]
    C0h = [torch.from_numpy(c).pin_memory() for c in C0host[args.warmup]]
    Coh = [torch.empty(c.shape, dtype=torch.float32).pin_memory() for c in C0h]
    rh = [torch.empty(X.shape[0], dtype=torch.int32).pin_memory() for X, _, _, _ in data]
    e2e = []
    for s in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n):
            Xs[i].copy_(Xh[i], non_blocking=True)
            if Xbh[i] is not None:
                Xbs[i].view(torch.int16).copy_(Xbh[i], non_blocking=True)
            C0buf[i].copy_(C0h[i], non_blocking=True)
        km.kmeans_solve_batched(ctx, Xs, C0buf, Couts, rhos, params=dict(m_max=10, max_iter=args.max_iter),
                                X_bf16s=Xbs)
        for i in range(n):
            Coh[i].copy_(Couts[i], non_blocking=True)
            rh[i].copy_(rhos[i], non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    h2d = sum(x.nbytes for x in Xh) + sum(b.nbytes for b in Xbh if b is not None) + sum(c.nbytes for c in C0h)
    d2h = sum(c.nbytes for c in Coh) + sum(r.nbytes for r in rh)

    lowd = [i for i, (X, _, _, _) in enumerate(data) if X.shape[1] <= 16]
    dense = [i for i in range(n) if i not in set(lowd)]
    loops = [max((inf[i]["iters"] for i in lowd), default=0) for inf in inf_aa]
    ngrp = len(groups)
    ham = any(inf[i]["scanned_rows"] < inf[i]["assign_passes"] * data[i][0].shape[0] for inf in inf_aa for i in lowd)
    mix = any(data[i][2] * data[i][0].shape[1] > 64 for i in lowd)
    launches = sum(batched_launches(L, ngrp, ham, mix, [(inf[i]["iters"], inf[i]["rejected"]) for i in dense])
                   for inf, L in zip(inf_aa, loops))
    E_aa = np.array([[inf[i]["E"] for i in range(n)] for inf in inf_aa])
    E_ll = np.array([[inf[i]["E"] for i in range(n)] for inf in inf_ll])
    line = {
        "metric": METRIC, "value": n * args.steps / tot_aa, "unit": "instance solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_aa / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 distances for d=64)",
        "data": "synthetic",
        "config": {"workload": "batched_512", "instances": n, "N": "log-U[1e3,2e5]", "d": "{2,3,16,64}",
                   "K": "log-U[8,256]", "m_max": 10, "max_iter": args.max_iter, "parallelism": "replicas x1",
                   "l2": "flushed before every step (256 MB write)",
                   "graph": "one graph per batch (recorded and tuned once); C0s copied into fixed buffers"},
        "p50_ms": pct(ms_aa, 50), "p99_ms": pct(ms_aa, 99),
        "aa": {"instance_solves_per_s": n * args.steps / tot_aa, "batch_ms_p50": pct(ms_aa, 50),
               "iters_mean": float(np.mean([[inf[i]["iters"] for i in range(n)] for inf in inf_aa])),
               "rejected_mean": float(np.mean([[inf[i]["rejected"] for i in range(n)] for inf in inf_aa]))},
        "lloyd": {"instance_solves_per_s": n * args.steps / tot_ll, "batch_ms_p50": pct(ms_ll, 50),
                  "iters_mean": float(np.mean([[inf[i]["iters"] for i in range(n)] for inf in inf_ll]))},
        "aa_over_lloyd_speed": tot_ll / tot_aa,
        "aa_lloyd_same_energy_frac": float(np.mean(np.abs(E_aa - E_ll) / E_ll <= 1e-6)),
        "tuning": desc,
        "roofline": roof,
        "e2e": {"value": n / statistics.median(e2e), "unit": "instance solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        import oracle
        idx = [i for i in lowd if data[i][0].shape[0] <= 20000][:12]
        t0 = time.perf_counter()
        for i in idx:
            X, _, K, ds = data[i]
            oracle.solve(X.astype(np.float64), C0host[0][i].astype(np.float64), m_max=10)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(idx) / dt, "unit": "instance solves/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"{len(idx)} low-d instances with N <= 20000 "
                                                            f"(Algorithm 1), solves/s over that sample"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_serving(args, rank, world, local_rank):
    """Poisson request stream through kmeans_server: p50/p99 latency and solves/s, AA vs Lloyd."""
    import torch
    import paper_1805_10638_gb300 as km

    torch.cuda.set_device(local_rank)
    reqs = datagen.serving_stream(args.serve_requests, rate=args.serve_rate, seed=7)
    # inputs in pinned host memory; the 2% large jobs share two data sets (their C0s differ)
    large_sets = []
    for j in range(2 if any(q["large"] for q in reqs) else 0):
        X = datagen.isotropic_mixture(4_000_000, 96, 4096, 70_000 + j, dtype=np.float32)
        large_sets.append((torch.from_numpy(X).pin_memory(),
                           torch.from_numpy(datagen.to_bf16_bits(X).view(np.int16)).pin_memory().view(torch.bfloat16)))
    # the small requests draw their data from a pool of at most 512 distinct data sets (request k takes
    # pool entry k mod 512 with its own C0), which bounds host memory and set-up time for 20,000 requests
    pool = {}
    inputs = []
    for k, q in enumerate(reqs):
        if q["large"]:
            Xt, Xbt = large_sets[k % len(large_sets)]
            C0 = datagen.init_centroids(Xt.numpy(), q["K"], q["data_seed"] + 1000)
            inputs.append((Xt, Xbt, torch.from_numpy(C0).pin_memory()))
        else:
            slot = k % 512
            if slot not in pool:
                X = datagen.isotropic_mixture(q["N"], q["d"], q["K"], q["data_seed"], dtype=np.float32)
                Xb = (torch.from_numpy(datagen.to_bf16_bits(X).view(np.int16)).pin_memory().view(torch.bfloat16)
                      if q["d"] > 16 else None)
                pool[slot] = (torch.from_numpy(X).pin_memory(), Xb, q["K"])
            Xt, Xb, K = pool[slot]
            C0 = datagen.init_centroids(Xt.numpy(), K, q["data_seed"] + 1000)
            inputs.append((Xt, Xb, torch.from_numpy(C0).pin_memory()))
    budget = int(args.serve_budget_gb * (1 << 30))

    def run(lloyd: bool, tscale: float = 1.0, nreq: int = 0):
        """Serve the stream (arrival times multiplied by tscale, the first nreq requests)."""
        srv = km.Server(local_rank, hbm_budget=budget, max_slots=512, max_large=args.serve_lanes)
        prm = dict(lloyd_only=1) if lloyd else dict(m_max=10)
        lat, nxt, inflight, iters, rejected, kind = [], 0, {}, [], [], []
        nr = nreq or len(reqs)
        t0 = time.perf_counter()
        while nxt < nr or inflight:
            now = time.perf_counter() - t0
            while nxt < nr and reqs[nxt]["t_arrival"] * tscale <= now:
                X, Xb, C0 = inputs[nxt]
                try:
                    inflight[srv.submit(X, C0, X_bf16=Xb, **prm)] = (nxt, reqs[nxt]["t_arrival"] * tscale)
                except km.KmeansError as e:       # a shape the server does not take: counted, not served
                    rejected.append((nxt, str(e)))
                nxt += 1
            srv.step()
            for t in list(inflight):
                res = srv.poll(t)
                if res is not None:
                    i, ta = inflight.pop(t)
                    lat.append((time.perf_counter() - t0) - ta)
                    kind.append("large" if reqs[i]["large"] else ("tensor" if reqs[i]["d"] > 16 else "lowd"))
                    iters.append(res[2]["iters"])
            if not inflight and nxt < nr:
                time.sleep(max(0.0, min(0.001, reqs[nxt]["t_arrival"] * tscale - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        by = {k: [l for l, c in zip(lat, kind) if c == k] for k in ("lowd", "tensor", "large")}
        return lat, wall, st, iters, rejected, by

    clocks = ClockSampler(local_rank)
    clocks.start()
    lat_aa, wall_aa, st_aa, it_aa, rej_aa, by_aa = run(False)
    lat_ll, wall_ll, st_ll, it_ll, rej_ll, by_ll = run(True)
    # sustainable rate: the same request sequence offered at lower rates (arrival times scaled);
    # a rate is sustained when the completions keep up with the arrivals (>= 97% of the offered
    # rate over the run) - then the backlog, and with it p99, stays bounded
    sweep = []
    for rate in [float(r) for r in args.serve_sweep.split(",") if r]:
        nreq = min(len(reqs), args.serve_sweep_requests)
        lat_s, wall_s, _, _, _, by_s = run(False, tscale=args.serve_rate / rate, nreq=nreq)
        span = reqs[nreq - 1]["t_arrival"] * args.serve_rate / rate
        sweep.append({"rate_per_s": rate, "requests": nreq, "solves_per_s": len(lat_s) / wall_s,
                      "keeps_up": len(lat_s) / wall_s >= 0.97 * nreq / span,
                      "p50_ms": 1e3 * pct(lat_s, 50), "p99_ms": 1e3 * pct(lat_s, 99),
                      "large_p99_ms": 1e3 * pct(by_s["large"], 99) if by_s["large"] else None})

    def classes(by):
        return {k: {"n": len(v), "p50_ms": 1e3 * pct(v, 50) if v else None, "p99_ms": 1e3 * pct(v, 99) if v else None}
                for k, v in by.items()}
    clk = clocks.stop()
    n = len(reqs)
    line = {
        "metric": METRIC, "value": len(lat_aa) / wall_aa, "unit": "solves/s", "n_gpus": world, "steps": n,
        "warmup": 0,
        "ms_per_step": 1e3 * wall_aa / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (bf16 distances for d > 16)", "data": "synthetic",
        "config": {"workload": "serving", "requests": n, "rate_per_s": args.serve_rate, "arrival_seed": 7,
                   "large_frac": 0.02, "large": "N=4e6, d=96, K=4096", "budget_gb": args.serve_budget_gb,
                   "max_slots": 512, "max_large": args.serve_lanes, "parallelism": "replicas x1",
                   "classes": "lowd = d <= 16 (continuous batch), tensor = d = 64 and large = N=4e6 (lanes)",
                   "data": "small requests cycle through 512 distinct data sets (own C0 each); large jobs share 2"},
        "p50_ms": 1e3 * pct(lat_aa, 50), "p99_ms": 1e3 * pct(lat_aa, 99),
        "aa": {"solves_per_s": len(lat_aa) / wall_aa, "p50_ms": 1e3 * pct(lat_aa, 50), "p99_ms": 1e3 * pct(lat_aa, 99),
               "iters_mean": float(np.mean(it_aa)), "steps": st_aa["steps"], "pool_peak_gb": st_aa["pool_peak"] / 2**30,
               "by_class": classes(by_aa)},
        "lloyd": {"solves_per_s": len(lat_ll) / wall_ll, "p50_ms": 1e3 * pct(lat_ll, 50), "p99_ms": 1e3 * pct(lat_ll, 99),
                  "iters_mean": float(np.mean(it_ll)), "steps": st_ll["steps"],
                  "pool_peak_gb": st_ll["pool_peak"] / 2**30, "by_class": classes(by_ll)},
        "latency": "arrival (wall clock) to results in host memory, including the host-to-device copy of X",
        "rate_sweep_aa": sweep,
        "sustainable_rate_per_s": max([w["rate_per_s"] for w in sweep if w["keeps_up"]], default=None),
        "rejected": len(rej_aa), "rejected_examples": [r for _, r in rej_aa[:3]],
        "e2e": {"value": len(lat_aa) / wall_aa, "unit": "solves/s",
                "h2d_bytes_per_step": int(np.mean([x.nbytes + (b.nbytes if b is not None else 0) + c.nbytes
                                                   for x, b, c in inputs])),
                "d2h_bytes_per_step": int(np.mean([c.nbytes + 4 * x.shape[0] for x, _, c in inputs]))},
        "roofline": None,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1805_10638_gb300 as km

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = dict(WORKLOADS[args.workload])
    if args.rows > 0:        # a profiler case, not a bench line: the JSON says so
        wl.update(N=args.rows, note="smaller case of the same generator for profiler captures; not a bench value")
    dense = wl["workload"] == "dense_1m"
    X, Xb = load_data(wl, args.rows)
    N, d, K = X.shape[0], X.shape[1], wl["K"]
    nsteps = args.steps + args.warmup
    C0s = [datagen.init_centroids(X, K, 1000 + s) for s in range(nsteps)]
    stream = torch.cuda.current_stream()
    ctx = km.Context(local_rank, stream=stream.cuda_stream)
    Xd = torch.from_numpy(X).cuda()
    Xbd = torch.from_numpy(Xb.view(np.int16)).cuda().view(torch.bfloat16) if dense else None
    # the low BF16 part of X (bf16(X - X_bf16)), supplied once like X_bf16
    Xld = (torch.from_numpy(datagen.to_bf16_bits(X - datagen.bf16_bits_to_f32(Xb)).view(np.int16)).cuda()
           if dense else None)
    C0d = [torch.from_numpy(c).cuda() for c in C0s]
    C_out = torch.empty((K, d), dtype=torch.float32, device="cuda")
    rho = torch.empty(N, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    solve_kw = dict(max_iter=args.max_iter)

    # the solver's graph is recorded once per buffer set: each step's C0 is copied into one
    # device buffer (outside the timed region) so that every step replays the same graph
    C0buf = torch.empty_like(C0d[0])

    def leg(lloyd: bool):
        kw = dict(solve_kw, **(dict(lloyd_only=1) if lloyd else dict(m_max=wl["m_max"])))
        for s in range(args.warmup):
            C0buf.copy_(C0d[s])
            km.kmeans_solve(ctx, Xd, C0buf, C_out, rho, X_bf16=Xbd, X_lo=Xld, **kw)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        infos = []
        for s in range(args.steps):
            flush.fill_(float(s))
            C0buf.copy_(C0d[args.warmup + s])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, info = km.kmeans_solve(ctx, Xd, C0buf, C_out, rho, X_bf16=Xbd, X_lo=Xld, **kw)
            e1.record(stream)
            evs.append((e0, e1))
            infos.append(info)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, infos

    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_aa, inf_aa = leg(False)
    ms_ll, inf_ll = leg(True)
    clk = clocks.stop()

    tot_aa = sum(ms_aa) / 1e3
    tot_ll = sum(ms_ll) / 1e3
    tot_aa, tot_ll = max_over_ranks([tot_aa, tot_ll], dist, "cuda")

    # ---- roofline of the dominant kernel: the assignment pass, timed standalone (CUDA events).
    # Low-d: the pass with its fused change count.  Dense: the call's centroid packing, the
    # tensor-core kernel and the FP32 rescoring of the near-tie rows (X's low part supplied).
    rho_prev = rho.clone()
    nch = torch.zeros((), dtype=torch.int64, device="cuda")
    akw = dict(X_bf16=Xbd, X_lo=Xld) if dense else dict(rho_prev=rho_prev, n_changed=nch)
    for _ in range(3):
        km.kmeans_assign(ctx, Xd, C_out, rho, **akw)
    torch.cuda.synchronize()
    reps = 20
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        km.kmeans_assign(ctx, Xd, C_out, rho, **akw)
    a1.record(stream)
    torch.cuda.synchronize()
    assign_ms = a0.elapsed_time(a1) / reps
    peaks = measured_peaks()
    if dense:
        work = 2.0 * N * K * d                # BF16 MMA flops of the distance contraction x.c
        achieved = work / (assign_ms * 1e-3) / 1e12
        peak = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"bound": "tensor", "kernel": "k_dense_assign (tcgen05, split BF16: 3 MMAs per K step, fused top-2) "
                                              "+ centroid packing + FP32 rescoring of near-tie rows",
                "unit": "TFLOP/s",
                "note": "algorithmic 2*N*K*d flops per assignment call (the split-BF16 kernel issues 3x that on "
                        "the tensor pipe) over the call's CUDA-event time; peak = measured cuBLAS BF16 burst "
                        "(MEASURED_PEAKS.json)"}
    else:
        # ALU work of a brute-force assignment pass: per (sample, centroid) pair d FMAs of the
        # score plus about two argmin operations (compare, select), one lane operation each
        work = float(N) * K * (d + 2)
        achieved = work / (assign_ms * 1e-3) / 1e12
        clock_mhz = 2070.0
        peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * clock_mhz * 1e6 / 1e12
        cal = calibrated_fp32_peak()
        roof = {"bound": "alu", "kernel": "k_pass_lowd<float,3> (assignment pass)",
                "unit": "Tlane-op/s",
                "note": "N*K*(d+2) lane operations per pass (d FMAs + ~2 argmin ops per sample-centroid "
                        "pair) over the launch's CUDA-event time; peak = 152 SMs x 128 FP32 lanes x 2070 MHz "
                        "(derived from unit counts and the maximum clock); peak_calibrated = measured FP32 FMA "
                        "rate (profiles/fp32_fma_peak.md)",
                "peak_calibrated": cal, "frac_calibrated": (achieved / cal) if cal else None}
    traffic = profiled_traffic("k_pass_lowd_lowd_2m.md" if not dense else "k_dense_assign_dense_1m.md")
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak, "traffic": traffic,
                 "assign_ms": assign_ms})

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timing
    Xh = torch.from_numpy(X).pin_memory()
    Xbh = torch.from_numpy(Xb.view(np.int16)).view(torch.bfloat16).pin_memory() if dense else None
    C0h = [torch.from_numpy(c).pin_memory() for c in C0s]
    Coh = torch.empty((K, d), dtype=torch.float32).pin_memory()
    rh = torch.empty(N, dtype=torch.int32).pin_memory()
    km.kmeans_solve_host(ctx, Xh, C0h[0], Coh, rh, X_bf16=Xbh, m_max=wl["m_max"], **solve_kw)
    e2e_t = []
    for s in range(args.steps):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        km.kmeans_solve_host(ctx, Xh, C0h[args.warmup + s], Coh, rh, X_bf16=Xbh, m_max=wl["m_max"], **solve_kw)
        e2e_t.append(time.perf_counter() - t0)
    e2e_tot = sum(e2e_t)
    (e2e_tot,) = max_over_ranks([e2e_tot], dist, "cuda")

    # the results of the first timed steps again (untimed), for their error against the oracle
    res_aa, res_ll = [], []
    if world == 1 and not args.no_cpu_baseline and rank == 0:
        for lloyd, res in ((False, res_aa), (True, res_ll)):
            kw = dict(solve_kw, **(dict(lloyd_only=1) if lloyd else dict(m_max=wl["m_max"])))
            for s in range(min(args.steps, 3)):
                C0buf.copy_(C0d[args.warmup + s])
                _, _, info = km.kmeans_solve(ctx, Xd, C0buf, C_out, rho, X_bf16=Xbd, X_lo=Xld, **kw)
                res.append((C_out.cpu().numpy().copy(), rho.cpu().numpy().copy(), info["E"], info))

    # our kernels in the timed Algorithm 1 solves (Hamerly bounds are on when a pass skipped rows)
    ham = (not dense) and any(i["scanned_rows"] < i["assign_passes"] * N for i in inf_aa)
    launches = sum(solve_launches(i["iters"], dense, ham, K * d <= 64, i["rejected"], dense_inc()) for i in inf_aa)
    if rank == 0:
        E_aa = np.array([i["E"] for i in inf_aa])
        E_ll = np.array([i["E"] for i in inf_ll])
        same_E = float(np.mean(np.abs(E_aa - E_ll) / E_ll <= 1e-6))
        speed_same, n_same = same_energy_speed(ms_aa, ms_ll, E_aa, E_ll)
        h2d = int(X.nbytes + (Xb.nbytes if dense else 0) + C0s[0].nbytes)
        line = {
            "metric": METRIC,
            "value": world * args.steps / tot_aa,
            "unit": "solves/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_aa / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "bf16" if dense else "f32",
            "data": "synthetic",
            "config": dict(wl, parallelism=f"replicas x{world}", max_iter=args.max_iter,
                           l2="flushed before every step (256 MB write); X stays resident in HBM",
                           graph="recorded once; each step's C0 is copied into the same device buffer"),
            "p50_ms": pct(ms_aa, 50), "p99_ms": pct(ms_aa, 99),
            "aa": {"solves_per_s": world * args.steps / tot_aa, "p50_ms": pct(ms_aa, 50), "p99_ms": pct(ms_aa, 99),
                   "iters_mean": float(np.mean([i["iters"] for i in inf_aa])),
                   "accepted_mean": float(np.mean([i["accepted"] for i in inf_aa])),
                   "rejected_mean": float(np.mean([i["rejected"] for i in inf_aa])),
                   "passes_mean": float(np.mean([i["assign_passes"] for i in inf_aa])),
                   "converged_frac": float(np.mean([i["converged"] for i in inf_aa])),
                   "rescored_rows_mean": float(np.mean([i["rescored_rows"] for i in inf_aa])),
                   "scanned_frac": float(np.mean([i["scanned_rows"] / max(1, i["assign_passes"] * N)
                                                  for i in inf_aa])),
                   "E_mean": float(E_aa.mean())},
            "lloyd": {"solves_per_s": world * args.steps / tot_ll, "p50_ms": pct(ms_ll, 50),
                      "p99_ms": pct(ms_ll, 99),
                      "iters_mean": float(np.mean([i["iters"] for i in inf_ll])),
                      "passes_mean": float(np.mean([i["assign_passes"] for i in inf_ll])),
                      "scanned_frac": float(np.mean([i["scanned_rows"] / max(1, i["assign_passes"] * N)
                                                     for i in inf_ll])),
                      "converged_frac": float(np.mean([i["converged"] for i in inf_ll])),
                      "E_mean": float(E_ll.mean())},
            "aa_over_lloyd_speed": tot_ll / tot_aa,
            "aa_lloyd_same_energy_frac": same_E,
            "aa_over_lloyd_speed_same_energy": speed_same,
            "same_energy_solves": n_same,
            "roofline": roof,
            "e2e": {"value": world * args.steps / e2e_tot, "unit": "solves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(K * d * 4 + N * 4)},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            line.update(cpu_leg(args, wl, X, C0s, inf_aa, res_aa, res_ll))
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_1m", choices=sorted(WORKLOADS) + ["batched_512", "serving"])
    ap.add_argument("--batch-instances", type=int, default=512)
    # the configured stream is 20,000 requests at 200/s; the GPU sustains about 20/s with the 2% large
    # jobs, so the default serves its first 1000 requests (minutes) and finds the sustainable rate
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-sweep", default="10,20,40",
                    help="comma-separated lower arrival rates for the sustainable-rate sweep")
    ap.add_argument("--serve-sweep-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-lanes", type=int, default=4)
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--rows", type=int, default=0,
                    help="profiler captures only: N rows of the workload's generator instead of its full size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-solves", type=int, default=2)
    args = ap.parse_args()
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched_512":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "serving":
        run_serving(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
