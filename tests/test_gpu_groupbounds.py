"""Group bounds (Yinyang-style) on the FP32 low-d solver passes.

Where Hamerly's half distances would cost O(K^2 d) per pass (K*K*d > 2^23) the standalone solver
keeps, per sample, one lower bound per group of nearby centroids (groups fixed from C^0 by Morton
order) and lowers each by its group's largest drift; KM_BOUNDS=group forces them at any K.  A row
keeps its label without a scan only when the bounds prove the assigned centroid the unique nearest
by a relative margin of 1e-5, so a solve with group bounds must be bitwise the solve that scans every
row (KM_HAMERLY=0): same centroids, labels, energies and counts, for Lloyd and Algorithm 1, across
the accelerated jumps and the reverts of Algorithm 1."""
import numpy as np
import pytest
import torch

import datagen
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("iters", "accepted", "rejected", "assign_passes", "converged", "m_final", "E", "status")


def _solve(X, C0, **p):
    ctx = km.Context(0)
    C, rho, info = km.kmeans_solve(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), **p)
    torch.cuda.synchronize()
    ctx.close()
    return C.cpu().numpy(), rho.cpu().numpy(), info


def _same(a, b):
    assert a[0].tobytes() == b[0].tobytes()
    assert np.array_equal(a[1], b[1])
    for f in FIELDS:
        assert a[2][f] == b[2][f], f


@pytest.mark.parametrize("shape", [(150_000, 3, 1024, 0), (100_000, 2, 1500, 1), (60_000, 4, 800, 2)])
@pytest.mark.parametrize("lloyd", [False, True])
def test_group_bounds_at_large_k_change_nothing(shape, lloyd, monkeypatch):
    """Group bounds at K = 800..1500: bitwise the brute-force solve, fewer rows scanned."""
    need_gpu()
    N, d, K, seed = shape
    X, C0 = datagen.batched_instance(N, d, K, 5100 + seed, dtype=np.float32)
    p = dict(lloyd_only=1) if lloyd else dict(m_max=10)
    monkeypatch.setenv("KM_BOUNDS", "group")
    with_b = _solve(X, C0, **p)
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = _solve(X, C0, **p)
    _same(with_b, without)
    assert with_b[2]["scanned_rows"] < 0.7 * without[2]["scanned_rows"], (with_b[2], without[2])


@pytest.mark.parametrize("shape", [(200_000, 3, 256, 4), (80_000, 8, 64, 5), (50_000, 16, 100, 6)])
def test_forced_group_bounds_change_nothing(shape, monkeypatch):
    need_gpu()
    N, d, K, seed = shape
    X, C0 = datagen.batched_instance(N, d, K, 5200 + seed, dtype=np.float32)
    monkeypatch.setenv("KM_BOUNDS", "group")
    with_b = _solve(X, C0, m_max=10)
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = _solve(X, C0, m_max=10)
    _same(with_b, without)


def test_group_bounds_on_anisotropic_mixture(monkeypatch):
    """The low-d workload's mixture at K = 1024 (Dirichlet weights, anisotropic clusters)."""
    need_gpu()
    X, C0 = datagen.lowd_2m(seed=3, N=400_000, K=1024)
    monkeypatch.setenv("KM_BOUNDS", "group")
    with_b = _solve(X, C0, m_max=10)
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = _solve(X, C0, m_max=10)
    _same(with_b, without)
    assert with_b[2]["scanned_rows"] < 0.5 * without[2]["scanned_rows"]
