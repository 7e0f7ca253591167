"""GPU parity of the dense path (BF16 tcgen05 distances, FP32 rescoring, sort-based update).

Assignments identical to the FP64 oracle wherever the oracle's top-2 gap exceeds
1e-6 * max(||x||^2, ||c_(1)||^2, ||c_(2)||^2); counts exact; centroids and energy within 1e-6.
"""
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


def dense_data(N, d, K, seed):
    X = datagen.full_cov_mixture(N, d, max(K, 2), seed)
    Xb = datagen.to_bf16_bits(X)
    C0 = datagen.init_centroids(X, K, seed + 1000)
    return X, Xb, C0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_bf16(bits):
    return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)


@pytest.mark.parametrize("N,d,K", [(20_000, 128, 1024), (9_999, 64, 300), (4_097, 96, 256), (1_000, 128, 7),
                                   (128, 64, 128), (33, 24, 5)])
def test_dense_assign_masked_parity(ctx, N, d, K):
    X, Xb, C0 = dense_data(N, d, K, seed=N + d + K)
    rho = km.kmeans_assign(ctx, dev(X), dev(C0), X_bf16=dev_bf16(Xb)).cpu().numpy()
    check_assignment(X, C0, rho, f"N={N} d={d} K={K}")


def test_dense_assign_n_changed_and_dmin(ctx):
    X, Xb, C0 = dense_data(8_000, 64, 50, seed=3)
    Xd, Xbd = dev(X), dev_bf16(Xb)
    r0 = km.kmeans_assign(ctx, Xd, dev(C0), X_bf16=Xbd)
    C1 = C0 + np.float32(0.5)
    nch = torch.zeros((), dtype=torch.int64, device="cuda")
    dmin = torch.empty(8_000, dtype=torch.float32, device="cuda")
    r1 = km.kmeans_assign(ctx, Xd, dev(C1), rho_prev=r0, n_changed=nch, dmin=dmin, X_bf16=Xbd)
    a0, a1 = r0.cpu().numpy(), r1.cpu().numpy()
    assert int(nch.item()) == int((a0 != a1).sum())
    ref = ((X.astype(np.float64) - C1.astype(np.float64)[a1]) ** 2).sum(1)
    np.testing.assert_allclose(dmin.cpu().numpy(), ref, rtol=1e-5)


@pytest.mark.parametrize("N,d,K", [(50_001, 128, 1000), (3_000, 32, 17)])
def test_dense_update_parity_deterministic(ctx, N, d, K):
    r = np.random.default_rng(N)
    X = (r.normal(size=(N, d)) * 3).astype(np.float32)
    rho = r.integers(0, K - 2, size=N).astype(np.int32)       # two empty clusters
    Cp = r.normal(size=(K, d)).astype(np.float32)
    Xd, rd, Cd = dev(X), dev(rho), dev(Cp)
    C1, n1 = km.kmeans_update(ctx, Xd, rd, K, Cd)
    C1 = C1.clone()
    C2, n2 = km.kmeans_update(ctx, Xd, rd, K, Cd)
    assert torch.equal(C1, C2) and torch.equal(n1, n2)
    Co, no = oracle.update(X, rho, K, Cp)
    np.testing.assert_array_equal(n1.cpu().numpy(), no)
    assert rel_err(C1.cpu().numpy(), Co) < 1e-6
    np.testing.assert_array_equal(C1.cpu().numpy()[no == 0], Cp[no == 0])


def test_dense_energy_parity(ctx):
    X, Xb, C0 = dense_data(30_000, 64, 100, seed=5)
    rho, _, _ = oracle.assign(X, C0)
    E = km.kmeans_energy(ctx, dev(X), dev(C0), dev(rho)).item()
    Eo = oracle.energy(X, C0, rho)
    assert abs(E - Eo) / Eo < 1e-6


@pytest.mark.parametrize("method", ["lloyd", "aa"])
def test_dense_solve_matches_oracle(ctx, method):
    X, Xb, C0 = dense_data(20_000, 64, 64, seed=7)
    kw = dict(lloyd_only=1) if method == "lloyd" else {}
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), X_bf16=dev_bf16(Xb), **kw)
    Ch, rh = C.cpu().numpy(), rho.cpu().numpy()
    assert info["converged"] == 1, info
    Eo_at = oracle.energy(X, Ch, rh)
    assert abs(info["E"] - Eo_at) / Eo_at < 1e-6
    Cm, _ = oracle.update(X, rh, Ch.shape[0], Ch)
    assert rel_err(Ch, Cm) < 1e-6
    check_assignment(X, Ch, rh, "fixed point")
    Co, ro, io = oracle.solve(X, C0, lloyd=(method == "lloyd"))
    assert abs(info["E"] - io["E"]) / io["E"] < 1e-6, (info, io)
    if method == "lloyd":
        assert info["iters"] == io["iters"], (info, io)


def test_dense_solve_repeatable_and_host(ctx):
    X, Xb, C0 = dense_data(10_000, 32, 40, seed=9)
    Xd, Xbd, Cd = dev(X), dev_bf16(Xb), dev(C0)
    C1, r1, i1 = km.kmeans_solve(ctx, Xd, Cd, X_bf16=Xbd)
    C1, r1 = C1.clone(), r1.clone()
    C2, r2, i2 = km.kmeans_solve(ctx, Xd, Cd, X_bf16=Xbd)
    assert torch.equal(C1, C2) and torch.equal(r1, r2)


@pytest.mark.slow
def test_dense_solve_full_size_sampled(ctx):
    """Full-size dense workload (N=1M, d=128, K=1024) in the bench's launch configuration, solved to
    convergence: sampled rows against the oracle at the solution, the fixed point and the energy."""
    X, Xb, C0 = datagen.dense_1m(seed=0)
    C, rho, info = km.kmeans_solve(ctx, dev(X), dev(C0), X_bf16=dev_bf16(Xb))
    assert info["converged"] == 1, info
    Ch, rh = C.cpu().numpy(), rho.cpu().numpy()
    idx = np.sort(np.random.default_rng(1).choice(X.shape[0], 4_000, replace=False))
    check_assignment(X[idx], Ch, rh[idx], "sampled rows at the solution")
    Cm, cnt = oracle.update(X, rh, Ch.shape[0], Ch)
    assert cnt.sum() == X.shape[0]
    assert rel_err(Ch, Cm) < 1e-6
    Eo = oracle.energy(X, Ch, rh)
    assert abs(info["E"] - Eo) / Eo < 1e-6


@pytest.mark.slow
def test_dense_full_size_against_the_oracles_solves(ctx):
    """Full-size dense workload from the benchmark's first C0 against the FP64 oracle's own solves
    (tests/golden/dense_1m_oracle.json, written by make_dense_1m.py): Lloyd takes the oracle's
    iterations and ends at its energy to 1e-6; Algorithm 1 ends within 1e-6 of the oracle's energy
    (reading R20: the reduced-precision trajectory may stop at a neighbouring fixed point)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "dense_1m_oracle.json")))
    X, Xb, C0 = datagen.dense_1m(seed=0)
    Xd, Xbd, Cd = dev(X), dev_bf16(Xb), dev(C0)
    _, _, il = km.kmeans_solve(ctx, Xd, Cd, X_bf16=Xbd, lloyd_only=1)
    assert il["converged"] == 1 and il["iters"] == g["lloyd"]["iters"], (il, g["lloyd"])
    assert abs(il["E"] - g["lloyd"]["E"]) <= 1e-6 * g["lloyd"]["E"]
    _, _, ia = km.kmeans_solve(ctx, Xd, Cd, X_bf16=Xbd, m_max=10)
    assert ia["converged"] == 1
    assert abs(ia["E"] - g["aa"]["E"]) <= 1e-6 * g["aa"]["E"], (ia, g["aa"])


@pytest.mark.parametrize("shape", [(20_000, 64, 64, 7), (30_000, 128, 300, 8), (12_000, 96, 1024, 9)])
@pytest.mark.parametrize("lloyd", [False, True])
def test_dense_bounds_change_nothing(shape, lloyd, monkeypatch):
    """Hamerly bounds on the tensor-core solver passes: a row keeps its label without the scan only
    when its bounds prove it by a relative margin far beyond FP32 rounding, so the solve is bitwise
    the one that scans every row (KM_HAMERLY=0), for Lloyd and for Algorithm 1."""
    need_gpu()
    N, d, K, seed = shape
    X, Xb, C0 = dense_data(N, d, K, seed)
    kw = dict(lloyd_only=1) if lloyd else dict(m_max=10)

    def run():
        c = km.Context(0)
        C, rho, info = km.kmeans_solve(c, dev(X), dev(C0), X_bf16=dev_bf16(Xb), **kw)
        torch.cuda.synchronize()
        out = (C.cpu().numpy(), rho.cpu().numpy(), info)
        c.close()
        return out

    with_b = run()
    monkeypatch.setenv("KM_HAMERLY", "0")
    without = run()
    assert with_b[0].tobytes() == without[0].tobytes()
    assert np.array_equal(with_b[1], without[1])
    for f in ("iters", "accepted", "rejected", "assign_passes", "converged", "E", "status"):
        assert with_b[2][f] == without[2][f], (f, with_b[2], without[2])


def _solve_fresh(X, Xb, C0, **kw):
    c = km.Context(0)
    C, rho, info = km.kmeans_solve(c, dev(X), dev(C0), X_bf16=dev_bf16(Xb), **kw)
    torch.cuda.synchronize()
    out = (C.cpu().numpy(), rho.cpu().numpy(), info)
    c.close()
    return out


@pytest.mark.parametrize("shape", [(20_000, 64, 64, 7), (30_000, 128, 300, 8), (12_000, 96, 1024, 9)])
def test_dense_incremental_update_paths_agree(shape, monkeypatch):
    """The incremental update of the tensor-core solver passes keeps the exact integer sums of the
    last partition and adds the rows whose label changed, or rebuilds them through the sorted chain.
    Both give the same integers, so the default (rebuild past a tenth of the rows changed), a
    rebuild every pass (KM_DINC=2) and the list after the first pass (KM_DINC=3) are bitwise the
    same solve, Algorithm 1's energy-driven decisions included."""
    need_gpu()
    N, d, K, seed = shape
    X, Xb, C0 = dense_data(N, d, K, seed)
    base = _solve_fresh(X, Xb, C0, m_max=10)
    for mode in ("2", "3"):
        monkeypatch.setenv("KM_DINC", mode)
        other = _solve_fresh(X, Xb, C0, m_max=10)
        assert base[0].tobytes() == other[0].tobytes(), mode
        assert np.array_equal(base[1], other[1]), mode
        for f in ("iters", "accepted", "rejected", "assign_passes", "converged", "E", "status"):
            assert base[2][f] == other[2][f], (mode, f, base[2], other[2])


@pytest.mark.parametrize("shape", [(20_000, 64, 64, 7), (30_000, 128, 300, 8)])
def test_dense_incremental_update_against_sorted_and_oracle(shape, monkeypatch):
    """The incremental update against the sorted update over every row (KM_DINC=0).  Lloyd takes
    no decision on the energy, so both visit the same partitions: equal labels and iterations,
    means and energies to rounding.  The incremental solves' energies (Eq. 1 from the integer sums,
    FP64) and means (Eq. 4) are those of their partitions in the FP64 oracle's arithmetic."""
    need_gpu()
    N, d, K, seed = shape
    X, Xb, C0 = dense_data(N, d, K, seed)
    inc_l = _solve_fresh(X, Xb, C0, lloyd_only=1)
    inc_a = _solve_fresh(X, Xb, C0, m_max=10)
    monkeypatch.setenv("KM_DINC", "0")
    srt_l = _solve_fresh(X, Xb, C0, lloyd_only=1)
    assert np.array_equal(inc_l[1], srt_l[1])
    for f in ("iters", "assign_passes", "converged", "status"):
        assert inc_l[2][f] == srt_l[2][f], (f, inc_l[2], srt_l[2])
    assert rel_err(inc_l[0], srt_l[0]) < 1e-6
    assert abs(inc_l[2]["E"] - srt_l[2]["E"]) <= 1e-7 * srt_l[2]["E"]
    for C, rho, info in (inc_l, inc_a):
        assert info["converged"] == 1, info
        Eo = oracle.energy(X, C, rho)
        assert abs(info["E"] - Eo) <= 1e-9 * Eo, (info["E"], Eo)
        Cm, _ = oracle.update(X, rho, K, C)
        assert rel_err(C, Cm) < 1e-6
