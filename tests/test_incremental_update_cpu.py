"""The arithmetic of the dense solver passes' incremental update, emulated in numpy on the CPU and
checked against the FP64 oracle (no GPU; the kernels are checked by tests/test_gpu_dense.py).

The update keeps, per cluster j, S_j = sum over its rows of round(x * 2^F) in 64-bit integers and
its size N_j, with F = 60 - ilogb(N max||x||) fixed for the solve.  A pass starts from the sums of
the last partition and adds the rows whose label changed; the means are 2^-F S_j / N_j (Eq. 4)
and the energy (Eq. 1) is sum_i ||x_i||^2 + sum_j (N_j ||c_j||^2 - 2 c_j . 2^-F S_j).
"""
import math

import numpy as np

import datagen
import oracle


def scale(N, xmax):
    if N * xmax <= 0.0:
        return 0
    F = 60 - (math.frexp(N * xmax)[1] - 1)        # frexp: v = m 2^e with 0.5 <= m < 1, ilogb = e - 1
    return max(-100, min(100, F))


def quantise(X, F):
    # x * 2^F is exact in FP32; the conversion rounds to nearest, ties to even (like __float2ll_rn)
    return np.rint(X.astype(np.float32) * np.float32(2.0 ** F)).astype(np.int64)


def sums(Q, rho, K):
    S = np.zeros((K, Q.shape[1]), dtype=np.int64)
    np.add.at(S, rho, Q)
    return S, np.bincount(rho, minlength=K).astype(np.int64)


def energy_from_sums(S, Nj, C, F, x2):
    C = C.astype(np.float64)
    return x2 + float(np.sum(C * (Nj[:, None] * C - 2.0 * np.ldexp(S.astype(np.float64), -F))))


def test_scale_bounds_the_sums():
    # every component of every row at +max||x|| in one cluster: the largest possible sum, and the
    # largest change of one (all rows leaving one cluster for another), stay below 2^62
    for N, xmax in [(1, 1.0), (1_000_000, 37.5), (4_000_000, 1e-3), (2 ** 31 - 1, 1e4), (10, 3e-30)]:
        F = scale(N, xmax)
        top = N * (xmax * 2.0 ** F + 0.5)
        assert 2 * top < 2.0 ** 62 + 1.0, (N, xmax, F)
        assert top >= 2.0 ** 58 or F == 100, (N, xmax, F)   # and the scale is not wasted


def test_carried_sums_equal_rebuilt_sums():
    X = datagen.full_cov_mixture(20_000, 64, 50, 3)
    rng = np.random.default_rng(5)
    K = 50
    F = scale(X.shape[0], float(np.sqrt((X.astype(np.float64) ** 2).sum(1)).max()) * (1 + 1e-5))
    Q = quantise(X, F)
    rho = rng.integers(0, K, size=X.shape[0])
    S, Nj = sums(Q, rho, K)
    for frac in (0.002, 0.05, 0.5):                 # passes with few and with many changed rows
        new = rho.copy()
        ch = rng.random(X.shape[0]) < frac
        new[ch] = rng.integers(0, K, size=int(ch.sum()))
        moved = np.nonzero(new != rho)[0]
        dS = np.zeros_like(S)
        np.add.at(dS, new[moved], Q[moved])
        np.subtract.at(dS, rho[moved], Q[moved])
        dN = np.bincount(new[moved], minlength=K) - np.bincount(rho[moved], minlength=K)
        S_full, N_full = sums(Q, new, K)
        assert np.array_equal(S + dS, S_full) and np.array_equal(Nj + dN, N_full)
        rho, S, Nj = new, S_full, N_full


def test_energy_and_means_from_sums_match_the_oracle():
    X = datagen.full_cov_mixture(30_000, 96, 40, 11)
    K = 40
    C0 = datagen.init_centroids(X, K, 1011)
    rho = oracle.assign(X, C0)[0]
    Xd = X.astype(np.float64)
    F = scale(X.shape[0], float(np.sqrt((Xd ** 2).sum(1)).max()) * (1 + 1e-5))
    S, Nj = sums(quantise(X, F), rho, K)
    x2 = float((Xd ** 2).sum())
    for C in (C0, oracle.update(X, rho, K, C0)[0]):
        Eo = oracle.energy(X, C, rho)
        assert abs(energy_from_sums(S, Nj, C, F, x2) - Eo) <= 1e-11 * Eo
    Cm, cnt = oracle.update(X, rho, K, C0)
    G = np.where(Nj[:, None] > 0, np.ldexp(S.astype(np.float64), -F) / np.maximum(Nj, 1)[:, None], C0)
    assert np.array_equal(cnt, Nj)
    assert np.max(np.abs(G - Cm)) <= 1e-12 * np.max(np.abs(Cm))
