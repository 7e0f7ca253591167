"""Step parity: one loop pass of Algorithm 1 on the GPU against one oracle pass started from the
same state.

The GPU solver runs T passes and exports its state (kmeans_solve_passes); the oracle runs pass
T+1 from that state (oracle.step, FP64) and the GPU runs it too (a solve of T+1 passes: the
passes are deterministic, so its first T equal the exported ones).  Compared: the decisions of
the pass (revert or accept, new m, convergence), P^{T+1} (exact on rows whose oracle top-2 gap
is clear of the rounding tolerance), the stored energy E^{T+1}, G^{T+1} and F^{T+1} (1e-6
relative in reduced precision), and the least squares of the pass: theta against the oracle's
Householder QR on the GPU's own history (1e-10) and the accelerated iterate
C^{T+2} = G - dG theta (Eq. 8, Algorithm 1's sign).  Workloads: FP64 small_2d, FP32 low-d with
K*d = 768, BF16 tensor-core path with K*d = 131,072.
"""
import math

import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_1805_10638_gb300 as km
from gpu_util import assignment_mask, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = km.Context(0)
    yield c
    c.close()


def _as_oracle_state(s):
    return dict(C=s["C"], CAU=s["C_AU"], F=s["F"], dF=s["dF"], dG=s["dG"], count=s["ring_count"],
                Pprev=s["rho"], t=s["t"], m=s["m"], from_lloyd=s["from_lloyd"], E_prev=s["E_prev"],
                E_prev2=s["E_prev2"], accepted=s["accepted"], rejected=s["rejected"], assign_passes=s["passes"])


def _check_step(ctx, X, C0, T, rtol, X_bf16=None, X64=None):
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C0).cuda()
    Xb = torch.from_numpy(X_bf16.view(np.int16)).cuda() if X_bf16 is not None else None
    sT = km.kmeans_solve_passes(ctx, Xd, Cd, T, X_bf16=Xb)
    s1 = km.kmeans_solve_passes(ctx, Xd, Cd, T + 1, X_bf16=Xb)
    assert not sT["done"], "pick T before convergence"
    X64 = np.asarray(X, np.float64) if X64 is None else X64
    o, rec = oracle.step(X64, _as_oracle_state(sT))
    E_ref = o["E_prev"] if not o["done"] else o["E"]
    # the pass's decisions are the oracle's unless a margin is within rounding of zero
    margins = [rec["margin_safe"], rec["margin_lo"], rec["margin_hi"]]
    near = any(np.isfinite(mg) and abs(mg) < 1e-6 * E_ref for mg in margins)
    if not near:
        assert s1["rejected"] - sT["rejected"] == rec["rejected"]
        assert s1["done"] == o["done"]
        assert s1["m"] == o["m"]
    # the assignment of the pass, at the centroids it used (C^{T+1}, or C_AU after a revert)
    C_used = sT["C_AU"] if rec["rejected"] else sT["C"]
    rho_o, _, gap_o = oracle.assign(X64, C_used)
    mask, _ = assignment_mask(X64, C_used, rho_o, gap_o)
    np.testing.assert_array_equal(o["Pprev"], rho_o)
    bad = np.nonzero(mask & (s1["rho"] != rho_o))[0]
    assert bad.size == 0, f"{bad.size} unmasked rows differ"
    if o["done"]:
        return rec
    # the update, residual and energy of the pass from the GPU's own assignment, in FP64 (Eq. 4, Eq. 1)
    K = C_used.shape[0]
    G_ref, _ = oracle.update(X64, s1["rho"], K, C_used)
    assert rel_err(s1["C_AU"], G_ref) <= rtol
    assert np.linalg.norm(s1["F"] - (G_ref - C_used)) <= rtol * np.linalg.norm(G_ref)
    E_ref = oracle.energy(X64, C_used, s1["rho"])
    assert abs(s1["E_prev"] - E_ref) <= rtol * E_ref
    # against the oracle's own pass: labels differ only on tie-band rows, the stored energy agrees
    assert int((s1["rho"] != o["Pprev"]).sum()) <= int((~mask).sum())
    assert abs(s1["E_prev"] - o["E_prev"]) <= rtol * o["E_prev"]
    # the newest differences (the rest of the ring is the input, shifted)
    assert s1["ring_count"] == o["count"]
    np.testing.assert_array_equal(s1["dF"][1:], sT["dF"][:s1["ring_count"] - 1])
    assert np.linalg.norm(s1["dG"][0] - (G_ref - sT["C_AU"]).ravel()) <= rtol * np.linalg.norm(G_ref)
    assert np.linalg.norm(s1["dF"][0] - (G_ref - C_used - sT["F"]).ravel()) <= rtol * np.linalg.norm(G_ref)
    # least squares of the pass on the GPU's own history: theta to 1e-10 against the oracle's QR
    mt = s1["m_t"]
    assert mt == min(o["m"], T + 1, o["count"])
    if mt > 0:
        th_o, rank_o = oracle.ls_qr(s1["dF"][:mt].T, s1["F"].ravel())
        assert s1["rank"] == rank_o
        th = s1["theta"][:mt]
        assert np.linalg.norm(th - th_o) <= 1e-10 * max(np.linalg.norm(th_o), 1e-300)
        # Eq. 8 with Algorithm 1's sign: C^{T+2} = G^{T+1} - sum_j theta_j dG_j
        C_next = s1["C_AU"].ravel() - s1["dG"][:mt].T @ th_o
        assert rel_err(s1["C"].ravel(), C_next) <= 1e-12
    return rec


@pytest.mark.parametrize("T", [2, 5, 9])
def test_step_fp64_small_2d(ctx, T):
    X, C0 = datagen.small_2d(seed=1)
    rec = _check_step(ctx, X, C0, T, rtol=1e-12)
    assert rec["t"] == T + 1


@pytest.mark.parametrize("T", [3, 12, 30])
def test_step_fp32_lowd_kd768(ctx, T):
    X, C0 = datagen.lowd_2m(seed=0, N=200_000, K=256)
    _check_step(ctx, X, C0, T, rtol=1e-6)


@pytest.mark.parametrize("T", [2, 6])
def test_step_bf16_dense_kd131072(ctx, T):
    X, Xb, C0 = datagen.dense_1m(seed=0, N=40_000, K=1024)
    _check_step(ctx, X, C0, T, rtol=1e-6, X_bf16=Xb)


def test_solve_passes_zero_is_the_prologue(ctx):
    """After the prologue: C = C_AU = G(C^0), F = C^1 - C^0, P^0 = Assign(C^0), t = 1 (Algorithm 1's
    first line)."""
    X, C0 = datagen.small_2d(seed=0)
    s = km.kmeans_solve_passes(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), 0)
    rho0, _, _ = oracle.assign(X, C0)
    G, _ = oracle.update(X, rho0, C0.shape[0], C0)
    np.testing.assert_array_equal(s["rho"], rho0)
    assert rel_err(s["C"], G) < 1e-14 and rel_err(s["C_AU"], G) < 1e-14
    assert np.abs(s["F"] - (G - C0)).max() < 1e-12
    assert (s["t"], s["from_lloyd"], s["ring_count"], s["m"]) == (1, 1, 0, 2)
    assert math.isinf(s["E_prev"])
