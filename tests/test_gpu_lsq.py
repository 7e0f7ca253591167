"""The device least squares of Eq. 7 (kmeans_lsq: the solver's routine on a given history) against
the oracle's Householder QR (oracle.ls_qr), on well- and ill-conditioned histories, and the
solver with the QR route forced against the golden FP64 counts."""
import json
import os

import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

QR, AUTO, GRAM = 1, 0, 2


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = km.Context(0)
    yield c
    c.close()


def _history(n, sv, seed):
    """[n, m] with the given singular values (newest column first) and a right-hand side."""
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.normal(size=(n, len(sv))))
    V, _ = np.linalg.qr(r.normal(size=(len(sv), len(sv))))
    A = (U * np.asarray(sv)) @ V.T
    return A, r.normal(size=n)


def _lsq(ctx, A, f, method, rank_tol=1e-12):
    dF = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    th, rank, qr = km.kmeans_lsq(ctx, dF, torch.from_numpy(f).cuda(), rank_tol=rank_tol, method=method)
    return th.cpu().numpy(), rank, qr


@pytest.mark.parametrize("n,m", [(20, 1), (768, 2), (768, 10), (4096, 16), (131072, 10), (3000, 30)])
def test_qr_matches_oracle_well_conditioned(ctx, n, m):
    A, f = _history(n, np.geomspace(1.0, 1e-2, m), seed=n + m)
    th_o, rank_o = oracle.ls_qr(A, f)
    for method in (QR, AUTO, GRAM):
        th, rank, qr = _lsq(ctx, A, f, method)
        assert rank == rank_o == m
        assert qr == (method == QR)                    # well conditioned: the Gram route certifies itself
        # Section 2.1's system through either route: equal to the oracle's QR to 1e-10 relative
        assert np.linalg.norm(th - th_o) <= 1e-10 * np.linalg.norm(th_o), (method, th, th_o)


@pytest.mark.parametrize("cond", [1e6, 1e9, 1e11])
def test_ill_conditioned_histories_keep_every_column(ctx, cond):
    """Condition numbers between 1e6 and 1e12 keep all columns under the 1e-12 cut; the solver's
    rule hands them to the QR (the Gram route cannot certify its factor there)."""
    m = 6
    A, _ = _history(768, np.geomspace(1.0, 1.0 / cond, m), seed=int(np.log10(cond)))
    theta_true = np.linspace(1.0, -2.0, m)
    f = A @ theta_true
    th_o, rank_o = oracle.ls_qr(A, f)
    tol = 1e-16 * cond * 50 * np.abs(theta_true).max()
    for method in (QR, AUTO):
        th, rank, qr = _lsq(ctx, A, f, method)
        assert rank == rank_o == m and qr == 1
        np.testing.assert_allclose(th, theta_true, rtol=0, atol=tol)
        np.testing.assert_allclose(th, th_o, rtol=0, atol=tol)


def test_rank_cut_drops_dependent_column(ctx):
    r = np.random.default_rng(11)
    A = r.normal(size=(500, 4))
    A[:, 3] = A[:, 0] - 0.5 * A[:, 2] + 1e-13 * r.normal(size=500)
    f = r.normal(size=500)
    th_o, rank_o = oracle.ls_qr(A, f)
    for method in (QR, AUTO):
        th, rank, qr = _lsq(ctx, A, f, method)
        assert rank == rank_o == 3 and th[3] == 0.0
        np.testing.assert_allclose(th[:3], th_o[:3], rtol=1e-9)
    # an exactly zero newest difference: rank 0 on every route
    for method in (QR, AUTO, GRAM):
        th, rank, _ = _lsq(ctx, np.zeros((50, 3)), r.normal(size=50), method)
        assert rank == 0 and not th.any()


def test_lsq_argument_errors(ctx):
    L = km.load()
    d = torch.zeros(4, device="cuda", dtype=torch.float64)
    assert L.kmeans_lsq(ctx.handle, None, 4, 1, d.data_ptr(), 1e-12, 0, d.data_ptr(), None, None) == 1
    assert L.kmeans_lsq(ctx.handle, d.data_ptr(), 4, 33, d.data_ptr(), 1e-12, 0, d.data_ptr(), None, None) == 1
    assert L.kmeans_lsq(ctx.handle, d.data_ptr(), 4, 1, d.data_ptr(), 1e-12, 3, d.data_ptr(), None, None) == 1
    assert L.kmeans_lsq(ctx.handle, d.data_ptr(), 0, 1, d.data_ptr(), 1e-12, 0, d.data_ptr(), None, None) == 1


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "small_2d.json")


@pytest.mark.parametrize("seed", range(5))
def test_solver_with_qr_route_matches_golden_counts(ctx, seed, monkeypatch):
    """KM_LSQ=qr makes every solver step take the Householder QR: FP64 counts stay bit-exact."""
    monkeypatch.setenv("KM_LSQ", "qr")
    g = json.load(open(GOLDEN))["seeds"][str(seed)]["aa"]
    X, C0 = datagen.small_2d(seed)
    C, rho, info = km.kmeans_solve(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), m_max=10)
    assert (info["iters"], info["accepted"], info["rejected"], info["assign_passes"]) == (
        g["iters"], g["accepted"], g["rejected"], g["assign_passes"])
    assert info["ls_qr_solves"] > 0
    err = np.linalg.norm(C.cpu().numpy() - np.array(g["C"])) / np.linalg.norm(np.array(g["C"]))
    assert err < 1e-12


def test_solver_qr_and_gram_routes_agree_in_fp32(ctx, monkeypatch):
    """Low-d FP32 solve (K*d = 768): the forced QR route and the default rule give the same solve."""
    X, C0 = datagen.lowd_2m(seed=2, N=100_000, K=256)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda()
    _, r0, i0 = km.kmeans_solve(ctx, Xd, Cd)
    monkeypatch.setenv("KM_LSQ", "qr")
    _, r1, i1 = km.kmeans_solve(ctx, Xd, Cd)
    assert i0["ls_qr_solves"] == 0 and i1["ls_qr_solves"] > 0
    assert i0["converged"] == i1["converged"] == 1
    assert abs(i0["E"] - i1["E"]) <= 1e-6 * i0["E"]
