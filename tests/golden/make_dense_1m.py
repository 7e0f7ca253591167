"""Write tests/golden/dense_1m_oracle.json: the FP64 oracle's full-size solves of the dense workload.

Calls only ``oracle`` and ``datagen``.  Workload: N=1,000,000, d=128, K=1024 full-covariance
mixture (data seed 0, the FP32 samples), C0 = 1024 distinct samples (seed 1000, the first step of
the benchmark); Lloyd and Algorithm 1 (m_max=10, m0=2, eps1=0.02, eps2=0.5, exact convergence).
Stored per solve: iteration, accepted, rejected and assignment-pass counts, m at the end, the final
energy, the norm and sum of the final centroids, and the energy after every loop pass.  The
benchmark's reference arm scales its full-size time per assignment pass by this solve's pass
count; the full-size dense GPU test compares its Lloyd solve with it.
Takes about an hour on 8 cores.  Run from the repository root:  python tests/golden/make_dense_1m.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402
import oracle   # noqa: E402


def main():
    X, _, C0 = datagen.dense_1m(seed=0)
    out = {"workload": "dense_1m N=1000000 d=128 K=1024, data seed 0, C0 seed 1000, fp64 oracle"}
    for name, kw in (("lloyd", dict(lloyd=True)), ("aa", dict(m_max=10))):
        t0 = time.time()
        C, rho, info, trace = oracle.solve(X, C0, trace=True, **kw)
        rec = dict(info)
        rec["C_norm"] = float(np.linalg.norm(C))
        rec["C_sum"] = float(C.sum())
        rec["E_trace"] = [r["E"] for r in trace]
        rec["seconds"] = round(time.time() - t0, 1)
        rec["threads"] = oracle.num_threads()
        out[name] = rec
        print(name, {k: v for k, v in rec.items() if k != "E_trace"}, flush=True)
    path = os.path.join(ROOT, "tests", "golden", "dense_1m_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
