"""Batched solves (kmeans_solve_batched) through the C ABI.

Every instance of a batch must give bitwise the results of kmeans_solve on it alone: the batched
kernels run each instance's blocks with the instance's own decomposition, and the launch shapes
picked by the autotuner change only the speed.  Standalone solves are checked against the FP64
oracle elsewhere; here one FP64 instance is also checked against the oracle directly.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("iters", "accepted", "rejected", "assign_passes", "converged", "m_final", "E", "status")


def _instances(n=24, seed=0):
    """Uneven instances: d in {2, 3, 16}, N in [1000, 40000], K in [4, 64], FP32 and FP64."""
    r = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(r.choice([2, 3, 16]))
        N = int(np.exp(r.uniform(np.log(1000), np.log(40000))))
        K = int(np.exp(r.uniform(np.log(4), np.log(64))))
        dt = np.float64 if i % 5 == 0 else np.float32
        X, C0 = datagen.batched_instance(N, d, K, 1000 + i, dtype=dt)
        lloyd = i % 3 == 0
        out.append((X, C0, dict(lloyd_only=1) if lloyd else dict(m_max=10)))
    return out


def _run_batch(ctx, inst):
    Xs = [torch.from_numpy(X).cuda() for X, _, _ in inst]
    C0s = [torch.from_numpy(C0).cuda() for _, C0, _ in inst]
    Cs, rhos, infos, st = km.kmeans_solve_batched(ctx, Xs, C0s, params=[p for _, _, p in inst])
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in Cs], [r.cpu().numpy() for r in rhos], infos


def _run_alone(ctx, inst):
    Cs, rhos, infos = [], [], []
    for X, C0, p in inst:
        C, rho, info = km.kmeans_solve(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), **p)
        torch.cuda.synchronize()
        Cs.append(C.cpu().numpy())
        rhos.append(rho.cpu().numpy())
        infos.append(info)
    return Cs, rhos, infos


def _same(a, b):
    Ca, ra, ia = a
    Cb, rb, ib = b
    for i in range(len(Ca)):
        assert Ca[i].tobytes() == Cb[i].tobytes(), f"instance {i}: centroids differ"
        assert np.array_equal(ra[i], rb[i]), f"instance {i}: assignments differ"
        for f in FIELDS:
            assert ia[i][f] == ib[i][f], f"instance {i}: {f} {ia[i][f]} != {ib[i][f]}"


def test_batched_equals_standalone():
    need_gpu()
    inst = _instances()
    ctx = km.Context(0)
    batch = _run_batch(ctx, inst)
    desc = km.batch_describe(ctx)
    alone = _run_alone(ctx, inst)
    _same(batch, alone)
    assert "grid" in desc
    for info in batch[2]:
        assert info["status"] == 0 and info["converged"] == 1


def test_batched_repeat_and_launch_modes(monkeypatch):
    need_gpu()
    inst = _instances(12, seed=1)
    ctx = km.Context(0)
    first = _run_batch(ctx, inst)
    _same(first, _run_batch(ctx, inst))            # cached graph
    monkeypatch.setenv("KM_GRAPH", "0")            # host loop, same kernels
    _same(first, _run_batch(ctx, inst))
    monkeypatch.setenv("KM_GRAPH", "1")
    monkeypatch.setenv("KM_TUNE", "0")             # default launch shapes
    ctx2 = km.Context(0)
    _same(first, _run_batch(ctx2, inst))


@pytest.mark.parametrize("variant", ["0", "1"])
def test_batched_kernel_variants_change_nothing(variant, monkeypatch):
    """The autotuner picks, per group of instances, the pass kernel's rows per thread (default or
    half) and its grid; forcing either variant gives bitwise the standalone solves."""
    need_gpu()
    inst = _instances(12, seed=2)
    monkeypatch.setenv("KM_BATCH_VARIANT", variant)
    ctx = km.Context(0)
    batch = _run_batch(ctx, inst)
    desc = km.batch_describe(ctx)
    assert f"-> variant {variant}" in desc or "f64" in desc, desc
    monkeypatch.delenv("KM_BATCH_VARIANT")
    _same(batch, _run_alone(km.Context(0), inst))


def test_batched_fp64_instance_matches_oracle():
    need_gpu()
    X, C0 = datagen.small_2d(seed=3)
    inst = [(X, C0, dict(m_max=10)), (X, C0, dict(lloyd_only=1))]
    Cs, rhos, infos = _run_batch(km.Context(0), inst)
    for (X_, C0_, p), C, rho, info in zip(inst, Cs, rhos, infos):
        C_ref, rho_ref, ref = oracle.solve(X_, C0_, lloyd=bool(p.get("lloyd_only", 0)))
        assert info["iters"] == ref["iters"]
        assert info["assign_passes"] == ref["assign_passes"]
        assert np.array_equal(rho, rho_ref)
        assert np.max(np.abs(C - C_ref)) <= 1e-12 * max(1.0, np.max(np.abs(C_ref)))


def test_batched_single_and_tiny_instances():
    need_gpu()
    r = np.random.default_rng(5)
    inst = []
    for N, d, K in [(1, 1, 1), (7, 2, 7), (33, 3, 1), (300, 16, 5)]:
        X = r.normal(size=(N, d)).astype(np.float32)
        inst.append((X, X[:K].copy(), dict(m_max=10)))
    ctx = km.Context(0)
    _same(_run_batch(ctx, inst), _run_alone(ctx, inst))


def test_batched_with_tensor_core_instances_equals_standalone():
    need_gpu()
    r = np.random.default_rng(11)
    inst = []
    for i in range(6):
        d = [3, 64, 2, 32, 16, 64][i]
        N = int(r.integers(3000, 20000))
        K = int(r.integers(8, 96))
        X, C0 = datagen.batched_instance(N, d, K, 3000 + i, dtype=np.float32)
        inst.append((X, C0, dict(m_max=10) if i % 2 else dict(lloyd_only=1)))
    ctx = km.Context(0)
    Xs = [torch.from_numpy(X).cuda() for X, _, _ in inst]
    Xbs = [torch.from_numpy(datagen.to_bf16_bits(X).view(np.int16)).cuda().view(torch.bfloat16)
           if X.shape[1] > 16 else None for X, _, _ in inst]
    C0s = [torch.from_numpy(C0).cuda() for _, C0, _ in inst]
    Cs, rhos, infos, _ = km.kmeans_solve_batched(ctx, Xs, C0s, params=[p for _, _, p in inst], X_bf16s=Xbs)
    torch.cuda.synchronize()
    for i, (X, C0, p) in enumerate(inst):
        C, rho, info = km.kmeans_solve(ctx, Xs[i], C0s[i], X_bf16=Xbs[i], **p)
        torch.cuda.synchronize()
        assert C.cpu().numpy().tobytes() == Cs[i].cpu().numpy().tobytes(), f"instance {i}"
        assert torch.equal(rho, rhos[i]), f"instance {i}"
        for f in FIELDS:
            assert info[f] == infos[i][f], f"instance {i}: {f}"


def test_batched_rejects_dense_instances():
    need_gpu()
    ctx = km.Context(0)
    X = torch.randn(1000, 64, device="cuda")
    with pytest.raises(km.KmeansError):
        km.kmeans_solve_batched(ctx, [X], [X[:8].clone()])


def test_batched_nonfinite_instance_reports_status():
    need_gpu()
    inst = _instances(3, seed=2)
    X = inst[1][0].copy()
    X[5, 0] = np.nan
    inst[1] = (X, inst[1][1], inst[1][2])
    ctx = km.Context(0)
    Xs = [torch.from_numpy(a).cuda() for a, _, _ in inst]
    C0s = [torch.from_numpy(c).cuda() for _, c, _ in inst]
    _, _, infos, st = km.kmeans_solve_batched(ctx, Xs, C0s, params=[p for _, _, p in inst], check=False)
    assert st == 5 and infos[1]["status"] == 5
    assert infos[0]["status"] == 0 and infos[2]["status"] == 0
