"""K-Means++ seeding on the GPU (kmeans_seed_pp) against the FP64 oracle, through the C ABI.

Both sides form the weights with the same separately rounded FP64 operations and draw with the
same uniforms, so the chosen rows agree row for row: they could only differ where u W falls
within rounding (about 1e-13 relative) of an interval edge, which none of these seeds does."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = km.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _both(ctx, X, K, seed):
    u = np.random.default_rng(seed).random(K)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    C, idx = km.kmeans_seed_pp(ctx, Xd, K, u)
    torch.cuda.synchronize()
    io, Co = oracle.kmeanspp(X.astype(np.float64), K, u)
    return C.cpu().numpy(), idx.cpu().numpy(), io, Co


@pytest.mark.parametrize("seed", range(3))
def test_seed_fp64_matches_oracle(ctx, seed):
    X, _ = datagen.small_2d(seed)
    C, idx, io, Co = _both(ctx, X, 10, 70 + seed)
    np.testing.assert_array_equal(idx, io)
    np.testing.assert_array_equal(C, Co)


def test_seed_fp32_matches_oracle(ctx):
    X, _ = datagen.lowd_2m(seed=1, N=200_000, K=64)
    C, idx, io, _ = _both(ctx, X, 64, 80)
    np.testing.assert_array_equal(idx, io)
    np.testing.assert_array_equal(C, X[idx])
    assert len(set(idx.tolist())) == 64


def test_seed_full_size_lowd_2m(ctx):
    X, _ = datagen.lowd_2m(seed=0)
    _, idx, io, _ = _both(ctx, X, 256, 81)
    np.testing.assert_array_equal(idx, io)


def test_seed_d128(ctx):
    X = datagen.full_cov_mixture(20_000, 128, 32, 3)
    C, idx, io, _ = _both(ctx, X, 32, 82)
    np.testing.assert_array_equal(idx, io)
    np.testing.assert_array_equal(C, X[idx])


def test_seed_edge_cases(ctx):
    X, _ = datagen.small_2d(0)
    _, idx, io, _ = _both(ctx, X, 1, 83)                         # K = 1: floor(u0 N)
    np.testing.assert_array_equal(idx, io)
    Xs = np.random.default_rng(4).normal(size=(12, 2))
    _, idx, io, _ = _both(ctx, Xs, 12, 84)                       # N = K: every row once
    assert sorted(idx.tolist()) == list(range(12))
    np.testing.assert_array_equal(idx, io)
    Xo = np.ones((50, 3))
    _, idx, io, _ = _both(ctx, Xo, 5, 85)                        # all weights 0: uniform rows
    np.testing.assert_array_equal(idx, io)


def test_seed_errors(ctx):
    X = torch.from_numpy(np.ones((10, 2))).cuda()
    with pytest.raises(km.KmeansError):
        km.kmeans_seed_pp(ctx, X, 2, [0.5, 1.0])                # u must be below 1
    with pytest.raises(km.KmeansError):
        km.kmeans_seed_pp(ctx, X, 11, np.zeros(11))             # K > N
