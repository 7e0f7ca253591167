"""FP32 FMA peak of this GPU, measured (kmeans_measure_fp32_fma), with the SM clock sampled during
the runs: the ALU roofline peak of the low-d assignment pass.

Usage: python -m paper_1805_10638_gb300.calibrate [--runs 5] [--iters 20000]
Prints one markdown table row per run and the best, in FMA lane operations per second (T/s).
"""
from __future__ import annotations

import argparse
import statistics
import subprocess
import time

from ._lib import measure_fp32_fma


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=5)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args()
    measure_fp32_fma(a.device, 1000)
    print("| run | kernel ms | FMA T/s | SM MHz (nvidia-smi, during the run) |")
    print("|---:|---:|---:|---:|")
    best = 0.0
    for r in range(a.runs):
        smi = subprocess.Popen(["nvidia-smi", f"--id={a.device}", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits",
                                "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        time.sleep(0.2)
        rate, ms = measure_fp32_fma(a.device, a.iters)
        smi.terminate()
        out, _ = smi.communicate(timeout=5)
        clk = [float(x) for x in out.split() if x.strip().replace(".", "").isdigit()]
        best = max(best, rate)
        print(f"| {r} | {ms:.2f} | {rate / 1e12:.2f} | {statistics.median(clk) if clk else float('nan'):.0f} |")
    print(f"\nbest: {best / 1e12:.2f} T FMA/s")


if __name__ == "__main__":
    main()
