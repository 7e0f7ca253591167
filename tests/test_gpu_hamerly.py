"""Hamerly bounds on the FP32 low-d solver passes.

A row keeps its label without a full scan only when its bounds show that the assigned centroid is
the unique nearest one by a relative margin far beyond FP32 rounding, so a solve with bounds must
be bitwise the same as the solve that scans every row (KM_HAMERLY=0): same centroids, labels,
energies and iteration counts, for Lloyd and for Algorithm 1, standalone and batched."""
import numpy as np
import pytest
import torch

import datagen
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(60_000, 2, 16, 0), (120_000, 3, 64, 1), (80_000, 8, 40, 2), (50_000, 16, 100, 3), (200_000, 3, 256, 4)]
FIELDS = ("iters", "accepted", "rejected", "assign_passes", "converged", "m_final", "E", "status")


def _solve(X, C0, **p):
    ctx = km.Context(0)
    C, rho, info = km.kmeans_solve(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), **p)
    torch.cuda.synchronize()
    return C.cpu().numpy(), rho.cpu().numpy(), info


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lloyd", [False, True])
def test_bounds_change_nothing(shape, lloyd, monkeypatch):
    need_gpu()
    N, d, K, seed = shape
    X, C0 = datagen.batched_instance(N, d, K, 4000 + seed, dtype=np.float32)
    p = dict(lloyd_only=1) if lloyd else dict(m_max=10)
    with_b = _solve(X, C0, **p)
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = _solve(X, C0, **p)
    assert with_b[0].tobytes() == without[0].tobytes()
    assert np.array_equal(with_b[1], without[1])
    for f in FIELDS:
        assert with_b[2][f] == without[2][f], f


def test_bounds_on_anisotropic_full_size_lloyd(monkeypatch):
    need_gpu()
    X, C0 = datagen.lowd_2m(seed=0)
    X = np.ascontiguousarray(X[:500_000])
    with_b = _solve(X, C0, lloyd_only=1)
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = _solve(X, C0, lloyd_only=1)
    assert with_b[0].tobytes() == without[0].tobytes()
    assert np.array_equal(with_b[1], without[1])
    assert with_b[2]["iters"] == without[2]["iters"]


def test_bounds_batched_equal(monkeypatch):
    need_gpu()
    inst = [datagen.batched_instance(N, d, K, 5000 + s, dtype=np.float32) for N, d, K, s in SHAPES[:4]]
    Xs = [torch.from_numpy(X).cuda() for X, _ in inst]
    C0s = [torch.from_numpy(C0).cuda() for _, C0 in inst]
    ctx = km.Context(0)
    a = km.kmeans_solve_batched(ctx, Xs, C0s, params=dict(m_max=10))
    torch.cuda.synchronize()
    monkeypatch.setenv("KM_HAMERLY", "0")
    b = km.kmeans_solve_batched(km.Context(0), Xs, C0s, params=dict(m_max=10))
    torch.cuda.synchronize()
    for i in range(len(inst)):
        assert torch.equal(a[0][i], b[0][i]) and torch.equal(a[1][i], b[1][i])
        for f in FIELDS:
            assert a[2][i][f] == b[2][i][f], f


@pytest.mark.parametrize("shape", [(300_000, 3, 1024, 7), (200_000, 2, 1500, 8), (120_000, 4, 700, 9)])
@pytest.mark.parametrize("cap", [None, "300"])
def test_bounds_at_large_k_in_queue_rounds(shape, cap, monkeypatch):
    """K*K*d up to 2^23: Hamerly's queue holds at most 4,096 rows per block (KM_HQ_CAP lowers it), so
    the INIT pass and any pass that queues more rows than that drains the queue in rounds; a thread
    that finds it full resumes at the same row.  Bitwise the brute-force solve, for both methods."""
    need_gpu()
    N, d, K, seed = shape
    X, C0 = datagen.batched_instance(N, d, K, 4100 + seed, dtype=np.float32)
    if cap:
        monkeypatch.setenv("KM_HQ_CAP", cap)
    for p in (dict(lloyd_only=1), dict(m_max=10)):
        with_b = _solve(X, C0, **p)
        monkeypatch.setenv("KM_HAMERLY", "0")
        without = _solve(X, C0, **p)
        monkeypatch.delenv("KM_HAMERLY")
        assert with_b[0].tobytes() == without[0].tobytes()
        assert np.array_equal(with_b[1], without[1])
        for f in FIELDS:
            assert with_b[2][f] == without[2][f], f
        assert with_b[2]["scanned_rows"] < 0.7 * without[2]["scanned_rows"], (with_b[2], without[2])
