"""Strategies for m, compared as in Section 3 ("Settings of m", Tab. 2): fixed m against the
dynamic rule of Section 2.2 started at the same m, plus Lloyd for reference and, optionally, the
rule's thresholds eps1 / eps2 varied around the paper's 0.02 / 0.5.

Every solve runs on the GPU through the library (``kmeans_solve``); this module only chooses the
parameters, times the calls with CUDA events and tabulates #Iter as accepted/total (Tab. 2's a/b),
the time per solve and the MSE E/N (reading R15).

    python -m paper_1805_10638_gb300.sweep --workload lowd_2m --seeds 3 [--eps-grid] [--json]

The CLI draws its inputs from the repository's seeded generators (``datagen``), run from the
repository root; ``sweep()`` takes any device arrays.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import _lib as km

# Section 3 runs Algorithm 1 with m-bar = 30 and m initialised to 2; Tab. 2 adds fixed m = 2, 5
# and the dynamic rule started at 5.
PAPER_M_MAX = 30


def tab2_strategies(m_values=(2, 5), m_max: int = PAPER_M_MAX):
    out = [("Lloyd", dict(lloyd_only=1))]
    for m in m_values:
        out.append((f"fixed m={m}", dict(m_init=m, m_max=m_max, fixed_m=1)))
        out.append((f"dynamic m0={m}", dict(m_init=m, m_max=m_max)))
    return out


def eps_strategies(pairs=((0.02, 0.5), (0.01, 0.5), (0.05, 0.5), (0.02, 0.3), (0.02, 0.7)), m_init: int = 2,
                   m_max: int = PAPER_M_MAX):
    return [(f"dynamic m0={m_init} eps1={e1} eps2={e2}", dict(m_init=m_init, m_max=m_max, eps1=e1, eps2=e2))
            for e1, e2 in pairs]


def sweep(ctx: km.Context, X, C0s, strategies, X_bf16=None):
    """Solve X from every initial C0 in C0s with every (name, params) strategy.

    Returns one dict per strategy: accepted and iterations summed over the initialisations, mean
    time per solve (ms), mean MSE (E/N), mean final m, and whether every solve converged."""
    N = X.shape[0]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rows = []
    for name, p in strategies:
        # one untimed solve first: the plan and its graph are built once per parameter set
        km.kmeans_solve(ctx, X, C0s[0], X_bf16=X_bf16, **p)
        torch.cuda.synchronize()
        acc = it = 0
        ms = mse = mfin = 0.0
        conv = True
        for C0 in C0s:
            e0.record()
            _, _, info = km.kmeans_solve(ctx, X, C0, X_bf16=X_bf16, **p)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            acc += info["accepted"]
            it += info["iters"]
            mse += info["E"] / N
            mfin += info["m_final"]
            conv &= info["converged"] == 1
        n = len(C0s)
        rows.append(dict(strategy=name, params=p, accepted=acc, iters=it, ms_per_solve=ms / n, mse=mse / n,
                         m_final_mean=mfin / n, converged=conv, solves=n))
    return rows


def format_table(rows) -> str:
    lines = ["| strategy | #Iter (accepted / total) | time per solve (ms) | MSE | final m (mean) |",
             "|---|---:|---:|---:|---:|"]
    for r in rows:
        lines.append(f"| {r['strategy']} | {r['accepted']} / {r['iters']} | {r['ms_per_solve']:.2f} | "
                     f"{r['mse']:.6g} | {r['m_final_mean']:.1f} |")
    return "\n".join(lines)


def _inputs(workload: str, seeds: int):
    import datagen  # the repository's seeded generators (run from the repository root)
    if workload == "lowd_2m":
        X, _ = datagen.lowd_2m(seed=0)
        K = 256
    elif workload == "small_2d":
        X, _ = datagen.small_2d(0)
        K = 10
    else:
        raise SystemExit(f"unknown workload {workload}")
    C0s = [datagen.init_centroids(X, K, 1000 + s) for s in range(seeds)]
    return X, C0s


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="lowd_2m", choices=["lowd_2m", "small_2d"])
    ap.add_argument("--seeds", type=int, default=3, help="initialisations per strategy")
    ap.add_argument("--m", type=int, nargs="+", default=[2, 5], help="m values of Tab. 2")
    ap.add_argument("--m-max", type=int, default=PAPER_M_MAX)
    ap.add_argument("--eps-grid", action="store_true", help="also vary eps1 / eps2 around 0.02 / 0.5")
    ap.add_argument("--json", action="store_true", help="one JSON line per strategy instead of a table")
    args = ap.parse_args(argv)
    X, C0s = _inputs(args.workload, args.seeds)
    ctx = km.Context(0)
    Xd = torch.from_numpy(X).cuda()
    C0d = [torch.from_numpy(c).cuda() for c in C0s]
    strategies = tab2_strategies(args.m, args.m_max)
    if args.eps_grid:
        strategies += eps_strategies(m_max=args.m_max)
    rows = sweep(ctx, Xd, C0d, strategies)
    if args.json:
        for r in rows:
            print(json.dumps(dict(r, workload=args.workload)))
    else:
        print(f"{args.workload}: N={X.shape[0]}, d={X.shape[1]}, K={C0s[0].shape[0]}, {args.seeds} initialisations")
        print(format_table(rows))
    ctx.close()


if __name__ == "__main__":
    main()
