"""Fixed-m strategy (Section 3, "Settings of m"; Tab. 2) on the GPU against the FP64 oracle.

FP64 path: iteration, acceptance and pass counts bit-exact, centroids and energy to 1e-12.
FP32 path: the oracle's energy to 1e-6 and a fixed point (reading R20)."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_1805_10638_gb300 as km
from gpu_util import check_assignment, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = km.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("m", [2, 5])
@pytest.mark.parametrize("seed", range(3))
def test_fixed_m_fp64_matches_oracle(ctx, seed, m):
    X, C0 = datagen.small_2d(seed)
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), m_init=m, m_max=10, fixed_m=1)
    Co, ro, io = oracle.solve(X, C0, m_init=m, m_max=10, fixed_m=1)
    for f in ("iters", "accepted", "rejected", "assign_passes", "converged", "m_final"):
        assert info[f] == io[f], (f, info, io)
    assert rel_err(C.cpu().numpy(), Co) < 1e-12
    np.testing.assert_array_equal(rho.cpu().numpy(), ro)
    assert abs(info["E"] - io["E"]) / io["E"] < 1e-12


def test_fixed_m0_is_lloyd_on_gpu(ctx):
    X, C0 = datagen.small_2d(1)
    Xd, Cd = dev(X), dev(C0)
    C1, r1, i1 = km.kmeans_solve(ctx, Xd, Cd, lloyd_only=1)
    C1, r1 = C1.clone(), r1.clone()
    C2, r2, i2 = km.kmeans_solve(ctx, Xd, Cd, m_init=0, fixed_m=1)
    assert torch.equal(C1, C2) and torch.equal(r1, r2)
    assert i1["iters"] == i2["iters"] and i1["E"] == i2["E"] and i2["accepted"] == 0


@pytest.mark.parametrize("m", [2, 5])
def test_fixed_m_fp32_lowd(ctx, m):
    X, C0 = datagen.lowd_2m(seed=3, N=100_000, K=64)
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), m_init=m, fixed_m=1)
    Ch, rh = C.cpu().numpy(), rho.cpu().numpy()
    assert info["converged"] == 1 and info["m_final"] == m
    Cm, _ = oracle.update(X, rh, C.shape[0], Ch)
    assert rel_err(Ch, Cm) < 1e-6
    check_assignment(X, Ch, rh, "fixed point")
    _, _, io = oracle.solve(X, C0, m_init=m, fixed_m=1)
    assert abs(info["E"] - io["E"]) / io["E"] < 1e-6, (info, io)


def test_fixed_m_batched_equals_standalone(ctx):
    inst = [datagen.batched_instance(N, d, K, 6100 + i, dtype=np.float32)
            for i, (N, d, K) in enumerate([(20_000, 2, 12), (35_000, 3, 40), (12_000, 16, 20)])]
    Xs = [dev(X) for X, _ in inst]
    C0s = [dev(C0) for _, C0 in inst]
    p = dict(m_init=5, fixed_m=1)
    Cb, rb, ib, _ = km.kmeans_solve_batched(ctx, Xs, C0s, params=p)
    torch.cuda.synchronize()
    for i in range(len(inst)):
        C, r, info = km.kmeans_solve(ctx, Xs[i], C0s[i], **p)
        assert torch.equal(C, Cb[i]) and torch.equal(r, rb[i])
        for f in ("iters", "accepted", "rejected", "m_final", "E"):
            assert info[f] == ib[i][f], f


# Section 3 runs with m-bar = 30: the history ring beyond 16 columns takes the shared-memory
# least-squares variant.
@pytest.mark.parametrize("seed", range(3))
def test_m_max_30_fp64_matches_oracle(ctx, seed):
    X, C0 = datagen.small_2d(seed)
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), m_max=30)
    Co, ro, io = oracle.solve(X, C0, m_max=30)
    for f in ("iters", "accepted", "rejected", "assign_passes", "converged", "m_final"):
        assert info[f] == io[f], (f, info, io)
    assert rel_err(C.cpu().numpy(), Co) < 1e-12
    np.testing.assert_array_equal(rho.cpu().numpy(), ro)


def test_fixed_m_20_fp64_fixed_point(ctx):
    # 20 history columns: rank truncation decisions may round differently from the oracle's QR,
    # so the bar is the solve's own consistency and the fixed point
    X, C0 = datagen.small_2d(1)
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), m_init=20, m_max=30, fixed_m=1)
    Ch, rh = C.cpu().numpy(), rho.cpu().numpy()
    assert info["converged"] == 1 and info["m_final"] == 20
    assert info["assign_passes"] == 1 + info["iters"] + info["rejected"]
    Cm, _ = oracle.update(X, rh, C.shape[0], Ch)
    assert rel_err(Ch, Cm) < 1e-13
    np.testing.assert_array_equal(oracle.assign(X, Ch)[0], rh)
    assert abs(info["E"] - oracle.energy(X, Ch, rh)) / info["E"] < 1e-12


def test_sweep_tool_small(ctx):
    from paper_1805_10638_gb300 import sweep
    X, _ = datagen.small_2d(0)
    C0s = [dev(datagen.init_centroids(X, 10, 1000 + s)) for s in range(2)]
    rows = sweep.sweep(ctx, dev(X), C0s, sweep.tab2_strategies(m_max=30) + sweep.eps_strategies()[:2])
    assert [r["strategy"] for r in rows][:5] == ["Lloyd", "fixed m=2", "dynamic m0=2", "fixed m=5", "dynamic m0=5"]
    assert all(r["converged"] and r["solves"] == 2 for r in rows)
    assert rows[0]["accepted"] == 0
    assert rows[1]["m_final_mean"] == 2 and rows[3]["m_final_mean"] == 5
    for r in rows:                                   # each row's figures are those of its solves
        tot = 0
        for C0 in C0s:
            tot += km.kmeans_solve(ctx, dev(X), C0, **r["params"])[2]["iters"]
        assert tot == r["iters"]
    assert "| fixed m=2 |" in sweep.format_table(rows)
