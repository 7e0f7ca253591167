"""Write tests/golden/small_2d.json: oracle results for the small FP64 workload.

Calls only ``oracle`` and ``datagen``.  Workload: N=10,000, d=2, K=10 isotropic mixture, seeds
0-4, C0 = 10 distinct samples (seed + 1000); Lloyd and Algorithm 1 (m_max=10, m0=2,
eps1=0.02, eps2=0.5, exact convergence).  Stored per seed: iteration counts, accepted / rejected
counts, assignment passes, the final energy and the final centroids.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import datagen  # noqa: E402
import oracle   # noqa: E402


def main():
    out = {"workload": "small_2d N=10000 d=2 K=10 fp64", "seeds": {}}
    for seed in range(5):
        X, C0 = datagen.small_2d(seed)
        rec = {}
        for name, kw in (("lloyd", dict(lloyd=True)), ("aa", dict(m_max=10))):
            C, rho, info = oracle.solve(X, C0, **kw)
            rec[name] = dict(info, C=C.tolist())
        out["seeds"][str(seed)] = rec
    path = os.path.join(ROOT, "tests", "golden", "small_2d.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
