"""Benchmark: K-Means solves/s to convergence, Anderson-accelerated vs plain Lloyd, on one GB300.

Default workload ``lowd_2m``: N = 2,000,000 samples, d = 3, K = 256, FP32, a mixture of 256
anisotropic Gaussians (axis std log-U[0.1, 2], centres U[0,100]^3, Dirichlet(1) weights).
``--workload dense_1m``: N = 1,000,000, d = 128, K = 1024, X in BF16 with the FP32 copy, 1024
full-covariance Gaussians (the tensor-core path).  One data set (seed 0); each step starts from
its own C0 (K distinct samples, seed 1000 + step).  A step is one full solve to convergence
(tol = 0, max_iter = 1000) through the C ABI with X resident in HBM; L2 is flushed (256 MB
write) before every step, outside the step's CUDA events.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (host cores, a
bounded row sample of the same workload, scaled to full-size solves/s).
Multi-GPU (torchrun): independent replicas per rank (no data-path collective), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
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


def load_data(wl):
    """(X f32, X_bf16 uint16 or None) of the workload."""
    if wl["workload"] == "dense_1m":
        X, Xb, _ = datagen.dense_1m(seed=wl["data_seed"])
        return X, Xb
    X, _ = datagen.lowd_2m(seed=wl["data_seed"])
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
            os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
            self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
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
def oracle_sample_solves(X, C0s, sample_rows: int, n: int, m_max: int, lloyd: bool = False):
    """Time the FP64 oracle on a row sample; returns (seconds per solve list, cores, rows)."""
    import oracle
    N = X.shape[0]
    r = np.random.default_rng(12345)
    idx = np.sort(r.choice(N, size=min(sample_rows, N), replace=False))
    Xs = np.ascontiguousarray(X[idx])
    times = []
    for i in range(n):
        C0 = C0s[i % len(C0s)]
        t0 = time.perf_counter()
        oracle.solve(Xs, C0, lloyd=lloyd, m_max=m_max)
        times.append(time.perf_counter() - t0)
    return times, oracle.num_threads(), len(idx)


def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    X, _ = load_data(wl)
    K = wl["K"]
    C0s = [datagen.init_centroids(X, K, 1000 + s) for s in range(max(1, args.steps))]
    rows = args.ref_sample_rows if args.ref_sample_rows else (100_000 if wl["d"] <= 16 else 10_000)
    scale = rows / X.shape[0]
    oracle_sample_solves(X, C0s, rows, max(1, args.warmup), wl["m_max"])
    times, cores, rows = oracle_sample_solves(X, C0s, rows, args.steps, wl["m_max"])
    full = [t / scale for t in times]        # per-solve time scaled to the full row count
    value = len(full) / sum(full)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(full) / len(full), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(wl, parallelism="cpu-oracle"),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} of {X.shape[0]} rows per solve (same d, K, init), "
                                   f"AA solve time scaled by {X.shape[0]}/{rows}"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": 1e3 * pct(full, 50), "p99_ms": 1e3 * pct(full, 99),
    }
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
    wl = WORKLOADS[args.workload]
    dense = wl["workload"] == "dense_1m"
    X, Xb = load_data(wl)
    N, d, K = X.shape[0], X.shape[1], wl["K"]
    nsteps = args.steps + args.warmup
    C0s = [datagen.init_centroids(X, K, 1000 + s) for s in range(nsteps)]
    stream = torch.cuda.current_stream()
    ctx = km.Context(local_rank, stream=stream.cuda_stream)
    Xd = torch.from_numpy(X).cuda()
    Xbd = torch.from_numpy(Xb.view(np.int16)).cuda().view(torch.bfloat16) if dense else None
    C0d = [torch.from_numpy(c).cuda() for c in C0s]
    C_out = torch.empty((K, d), dtype=torch.float32, device="cuda")
    rho = torch.empty(N, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    solve_kw = dict(max_iter=args.max_iter)

    def leg(lloyd: bool):
        kw = dict(solve_kw, **(dict(lloyd_only=1) if lloyd else dict(m_max=wl["m_max"])))
        for s in range(args.warmup):
            km.kmeans_solve(ctx, Xd, C0d[s], C_out, rho, X_bf16=Xbd, **kw)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        infos = []
        for s in range(args.steps):
            flush.fill_(float(s))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, info = km.kmeans_solve(ctx, Xd, C0d[args.warmup + s], C_out, rho, X_bf16=Xbd, **kw)
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
    if dist:
        t = torch.tensor([tot_aa, tot_ll], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_aa, tot_ll = float(t[0]), float(t[1])

    # ---- roofline of the dominant kernel: the assignment pass, timed standalone (CUDA events)
    rho_prev = rho.clone()
    nch = torch.zeros((), dtype=torch.int64, device="cuda")
    for _ in range(3):
        km.kmeans_assign(ctx, Xd, C_out, rho, rho_prev=rho_prev, n_changed=nch, X_bf16=Xbd)
    torch.cuda.synchronize()
    reps = 20
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        km.kmeans_assign(ctx, Xd, C_out, rho, rho_prev=rho_prev, n_changed=nch, X_bf16=Xbd)
    a1.record(stream)
    torch.cuda.synchronize()
    assign_ms = a0.elapsed_time(a1) / reps
    flops = 2.0 * N * K * d                   # the distance contraction x.c
    achieved = flops / (assign_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    if dense:
        peak = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"bound": "tensor", "kernel": "k_dense_assign (tcgen05 BF16 + fused top-2) + rescoring",
                "note": "2*N*K*d BF16 MMA flops per assignment call over its CUDA-event time; peak = "
                        "measured cuBLAS BF16 burst (MEASURED_PEAKS.json)"}
        tkey = "k_dense_assign"
    else:
        clock_mhz = 2070.0
        peak = 2.0 * SM_COUNT_NOMINAL * FP32_LANES_PER_SM * clock_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "k_pass_lowd<float,3> (assignment pass)",
                "note": "2*N*K*d FP32 FMA flops per pass over the launch's CUDA-event time; peak = FP32 "
                        "FMA pipe 152 SMs x 128 lanes x 2 flops x 2070 MHz (derived, not measured)"}
        tkey = "k_pass_lowd<float,3>"
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get(tkey)
        except Exception:
            traffic = None
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": traffic, "assign_ms": assign_ms})

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
    if dist:
        t = torch.tensor([e2e_tot], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t[0])

    # our kernels per solve: dense 13 (prologue) + 17 per loop pass + 6 (epilogue);
    # low-d with the accelerated iterate fused into the update kernel 3 + 3 per pass + 2
    launches = sum((19 + 17 * i["iters"]) if dense else (5 + 3 * i["iters"]) for i in inf_aa)
    if rank == 0:
        E_aa = np.array([i["E"] for i in inf_aa])
        E_ll = np.array([i["E"] for i in inf_ll])
        same_E = float(np.mean(np.abs(E_aa - E_ll) / E_ll <= 1e-6))
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
                           l2="flushed before every step (256 MB write); X stays resident in HBM"),
            "p50_ms": pct(ms_aa, 50), "p99_ms": pct(ms_aa, 99),
            "aa": {"solves_per_s": world * args.steps / tot_aa, "p50_ms": pct(ms_aa, 50), "p99_ms": pct(ms_aa, 99),
                   "iters_mean": float(np.mean([i["iters"] for i in inf_aa])),
                   "accepted_mean": float(np.mean([i["accepted"] for i in inf_aa])),
                   "rejected_mean": float(np.mean([i["rejected"] for i in inf_aa])),
                   "passes_mean": float(np.mean([i["assign_passes"] for i in inf_aa])),
                   "converged_frac": float(np.mean([i["converged"] for i in inf_aa])),
                   "rescored_rows_mean": float(np.mean([i["rescored_rows"] for i in inf_aa])),
                   "E_mean": float(E_aa.mean())},
            "lloyd": {"solves_per_s": world * args.steps / tot_ll, "p50_ms": pct(ms_ll, 50),
                      "p99_ms": pct(ms_ll, 99),
                      "iters_mean": float(np.mean([i["iters"] for i in inf_ll])),
                      "passes_mean": float(np.mean([i["assign_passes"] for i in inf_ll])),
                      "converged_frac": float(np.mean([i["converged"] for i in inf_ll])),
                      "E_mean": float(E_ll.mean())},
            "aa_over_lloyd_speed": tot_ll / tot_aa,
            "aa_lloyd_same_energy_frac": same_E,
            "roofline": roof,
            "e2e": {"value": world * args.steps / e2e_tot, "unit": "solves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(K * d * 4 + N * 4)},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            rows = args.cpu_sample_rows if args.cpu_sample_rows else (200_000 if d <= 16 else 10_000)
            times, cores, rows = oracle_sample_solves(X, C0s, rows, args.cpu_solves, wl["m_max"])
            full = [t * X.shape[0] / rows for t in times]
            line["cpu_baseline"] = {"value": len(full) / sum(full), "unit": "solves/s", "cores": cores,
                                    "kind": "oracle",
                                    "sample": f"{len(times)} AA solves on {rows} of {X.shape[0]} rows "
                                              f"(same d, K, inits), time scaled by {X.shape[0]}/{rows}"}
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
    ap.add_argument("--workload", default="lowd_2m", choices=sorted(WORKLOADS))
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-rows", type=int, default=0)
    ap.add_argument("--cpu-solves", type=int, default=3)
    ap.add_argument("--ref-sample-rows", type=int, default=0)
    args = ap.parse_args()
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
