"""Seeded synthetic inputs for the K-Means workloads (shared by the oracle tests and the GPU path).

This module holds no K-Means arithmetic: it only draws Gaussian-mixture samples and initial
centroids with numpy's PCG64 (``numpy.random.default_rng(seed)``).  The mixtures stand in for
the paper's UCI/Birch datasets (Table 1), which are not available here; their shapes follow the
paper's range (d = 2..561, N = 7k..4.9M, K = 10..1000).

Workloads (sizes as named):

* ``small_2d``      N=10,000,  d=2,   K=10,   FP64.  10 isotropic sigma=1 Gaussians, centres
                    U[-10,10]^2, equal weights.
* ``lowd_2m``       N=2,000,000, d=3, K=256,  FP32.  256 axis-aligned Gaussians, per-axis std
                    log-U[0.1,2], centres U[0,100]^3, Dirichlet(1) weights (multinomial counts).
* ``dense_1m``      N=1,000,000, d=128, K=1024.  1024 Gaussians, centres N(0,4I), covariance
                    Q diag(lambda) Q^T with Haar Q and lambda log-U[0.01,1], equal weights.
                    FP32 X plus its BF16 copy (round to nearest even).
* ``batched_512``   512 instances, N log-U[1e3,2e5], d in {2,3,16,64}, K log-U[8,256],
                    FP32, each an isotropic mixture as ``small_2d`` scaled to its d and K.
* ``serving``       Poisson arrivals (rate 200/s, arrival seed 7): 98% instances shaped like
                    ``batched_512``, 2% large jobs N=4e6, d=96, K=4096 (isotropic sigma=1,
                    centres U[-10,10]^96).

Rows are shuffled so that cluster membership is not sorted.  Initial centroids are K distinct
samples drawn without replacement with seed ``data_seed + 1000``.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def isotropic_mixture(N: int, d: int, K: int, seed: int, sigma: float = 1.0,
                      lo: float = -10.0, hi: float = 10.0, dtype=np.float64) -> np.ndarray:
    """N samples of K equal-weight isotropic Gaussians (std sigma), centres U[lo,hi]^d."""
    r = _rng(seed)
    centres = r.uniform(lo, hi, size=(K, d))
    labels = r.integers(0, K, size=N)
    X = centres[labels] + sigma * r.standard_normal(size=(N, d))
    return X.astype(dtype)


def init_centroids(X: np.ndarray, K: int, seed: int) -> np.ndarray:
    """K distinct rows of X chosen without replacement (seeded); same dtype as X."""
    r = _rng(seed)
    idx = r.choice(X.shape[0], size=K, replace=False)
    idx.sort()
    return np.ascontiguousarray(X[idx])


def small_2d(seed: int = 0):
    """(X f64[10000,2], C0 f64[10,2])."""
    X = isotropic_mixture(10_000, 2, 10, seed)
    return X, init_centroids(X, 10, seed + 1000)


def anisotropic_mixture(N: int, d: int, K: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Axis-aligned Gaussians: std per axis log-U[0.1,2], centres U[0,100]^d, Dirichlet(1)
    weights realised as multinomial counts; rows shuffled."""
    r = _rng(seed)
    centres = r.uniform(0.0, 100.0, size=(K, d))
    scales = np.exp(r.uniform(np.log(0.1), np.log(2.0), size=(K, d)))
    w = r.dirichlet(np.ones(K))
    counts = r.multinomial(N, w)
    labels = np.repeat(np.arange(K), counts)
    r.shuffle(labels)
    X = np.empty((N, d), dtype=np.float64)
    chunk = 1 << 20
    for s in range(0, N, chunk):
        lab = labels[s:s + chunk]
        X[s:s + chunk] = centres[lab] + scales[lab] * r.standard_normal(size=(lab.shape[0], d))
    return X.astype(dtype)


def lowd_2m(seed: int = 0, N: int = 2_000_000, d: int = 3, K: int = 256):
    """(X f32[N,d], C0 f32[K,d]) for the low-dimensional workload."""
    X = anisotropic_mixture(N, d, K, seed)
    return X, init_centroids(X, K, seed + 1000)


def to_bf16_bits(X32: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (nearest, ties to even); returns the uint16 bit patterns."""
    u = np.ascontiguousarray(X32, dtype=np.float32).view(np.uint32)
    bias = ((u >> 16) & 1) + np.uint32(0x7FFF)
    return ((u + bias) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32)


def full_cov_mixture(N: int, d: int, K: int, seed: int) -> np.ndarray:
    """Equal-weight Gaussians, centres N(0,4I), covariance Q diag(lambda) Q^T (Haar Q,
    lambda log-U[0.01,1]); FP32, rows shuffled."""
    r = _rng(seed)
    centres = 2.0 * r.standard_normal(size=(K, d))
    labels = r.integers(0, K, size=N)
    order = np.argsort(labels, kind="stable")
    counts = np.bincount(labels, minlength=K)
    X = np.empty((N, d), dtype=np.float32)
    pos = 0
    for j in range(K):
        n = int(counts[j])
        Z = r.standard_normal(size=(d, d))
        Q, R = np.linalg.qr(Z)
        Q = Q * np.sign(np.diag(R))          # Haar-distributed orthogonal matrix
        lam = np.exp(r.uniform(np.log(0.01), np.log(1.0), size=d))
        A = Q * np.sqrt(lam)                 # x = mu + Q diag(sqrt(lam)) z
        z = r.standard_normal(size=(n, d))
        X[order[pos:pos + n]] = (centres[j] + z @ A.T).astype(np.float32)
        pos += n
    return X


def dense_1m(seed: int = 0, N: int = 1_000_000, d: int = 128, K: int = 1024):
    """(X f32[N,d], X_bf16 uint16[N,d], C0 f32[K,d]) for the dense workload."""
    X = full_cov_mixture(N, d, K, seed)
    return X, to_bf16_bits(X), init_centroids(X, K, seed + 1000)


def batched_shapes(n_inst: int = 512, seed: int = 0):
    """List of (N, d, K, data_seed) for the uneven batched workload."""
    r = _rng(seed + 500)
    Ns = np.exp(r.uniform(np.log(1e3), np.log(2e5), size=n_inst)).astype(np.int64)
    ds = r.choice(np.array([2, 3, 16, 64]), size=n_inst)
    Ks = np.exp(r.uniform(np.log(8), np.log(256), size=n_inst)).astype(np.int64)
    return [(int(Ns[i]), int(ds[i]), int(Ks[i]), int(seed * 100_000 + i)) for i in range(n_inst)]


def batched_instance(N: int, d: int, K: int, data_seed: int, dtype=np.float32):
    """(X, C0) of one batched instance: isotropic mixture as ``small_2d`` scaled to d and K."""
    X = isotropic_mixture(N, d, K, data_seed, dtype=dtype)
    return X, init_centroids(X, K, data_seed + 1000)


def serving_stream(n_req: int = 20_000, rate: float = 200.0, seed: int = 7,
                   large_frac: float = 0.02):
    """List of dicts {t_arrival, N, d, K, data_seed, large} for the request stream."""
    r = _rng(seed)
    gaps = r.exponential(1.0 / rate, size=n_req)
    t = np.cumsum(gaps)
    large = r.random(n_req) < large_frac
    shapes = batched_shapes(n_req, seed=seed)
    out = []
    for i in range(n_req):
        if large[i]:
            N, d, K = 4_000_000, 96, 4096
        else:
            N, d, K, _ = shapes[i]
        out.append(dict(t_arrival=float(t[i]), N=N, d=d, K=K, data_seed=int(seed * 1_000_000 + i),
                        large=bool(large[i])))
    return out
