"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test fixes a part of the oracle with an independent check: brute force in plain Python on
tiny inputs, a library routine (numpy bincount / lstsq / cholesky), a closed form, an invariant
the paper states, or a worked example derived by hand from Eq. 3, Eq. 4, Eq. 7 and Algorithm 1.
"""
import math

import numpy as np
import pytest

import datagen
import oracle


# ----------------------------------------------------------------------------- assignment, Eq. 3
def _brute_assign(X, C):
    rho, dmin, gap = [], [], []
    for x in X.tolist():
        ds = []
        for c in C.tolist():
            ds.append(sum((a - b) ** 2 for a, b in zip(x, c)))
        j = min(range(len(ds)), key=lambda k: (ds[k], k))
        s = sorted(ds)
        rho.append(j)
        dmin.append(ds[j])
        gap.append(s[1] - s[0] if len(s) > 1 else math.inf)
    return np.array(rho), np.array(dmin), np.array(gap)


@pytest.mark.parametrize("seed", range(6))
def test_assign_matches_brute_force(seed):
    r = np.random.default_rng(seed)
    N, K, d = int(r.integers(1, 64)), int(r.integers(1, 9)), int(r.integers(1, 4))
    X = r.normal(size=(N, d))
    C = r.normal(size=(K, d))
    if K >= 3:                      # adversarial ties: duplicated centroids
        C[K - 1] = C[1]
        C[2] = C[0]
    rho, dmin, gap = oracle.assign(X, C)
    brho, bdmin, bgap = _brute_assign(X, C)
    np.testing.assert_array_equal(rho, brho)
    np.testing.assert_allclose(dmin, bdmin, rtol=1e-13, atol=0)
    np.testing.assert_allclose(gap, bgap, rtol=1e-12, atol=1e-14)


def test_assign_integer_grid_ties_lowest_index():
    # points exactly half-way between integer centroids: squared distances tie exactly
    X = np.array([[0.5], [1.5], [2.5], [1.0]])
    C = np.array([[0.0], [1.0], [2.0], [3.0]])
    rho, _, gap = oracle.assign(X, C)
    np.testing.assert_array_equal(rho, [0, 1, 2, 1])
    assert gap[0] == 0.0 and gap[1] == 0.0 and gap[2] == 0.0


def test_assign_special_cases():
    X = np.random.default_rng(3).normal(size=(40, 3))
    rho, _, gap = oracle.assign(X, X[:1])
    assert (rho == 0).all() and np.isinf(gap).all()
    rho, dmin, _ = oracle.assign(X, X)           # K = N distinct centroids
    np.testing.assert_array_equal(rho, np.arange(40))
    assert oracle.energy(X, X, rho) == 0.0 and (dmin == 0).all()


# --------------------------------------------------------------------------------- update, Eq. 4
def test_update_matches_bincount_and_keeps_empty():
    r = np.random.default_rng(1)
    N, K, d = 500, 7, 3
    X = r.normal(size=(N, d))
    rho = r.integers(0, K - 2, size=N).astype(np.int32)   # clusters K-2, K-1 empty
    Cp = r.normal(size=(K, d))
    C, counts = oracle.update(X, rho, K, Cp)
    bc = np.bincount(rho, minlength=K)
    np.testing.assert_array_equal(counts, bc)
    assert counts.sum() == N
    for k in range(d):
        s = np.bincount(rho, weights=X[:, k], minlength=K)
        nz = bc > 0
        np.testing.assert_allclose(C[nz, k], s[nz] / bc[nz], rtol=1e-13)
    np.testing.assert_array_equal(C[bc == 0], Cp[bc == 0])


# --------------------------------------------------------------------------------- energy, Eq. 1
def test_energy_is_min_over_assignments():
    r = np.random.default_rng(2)
    X = r.normal(size=(300, 2))
    C = r.normal(size=(5, 2))
    rho, dmin, _ = oracle.assign(X, C)
    E = oracle.energy(X, C, rho)
    assert E == pytest.approx(math.fsum(dmin.tolist()), rel=1e-13)
    # surrogate property (Eq. 5): any other assignment gives an energy >= E(C)
    for s in range(5):
        other = np.random.default_rng(10 + s).integers(0, 5, size=300).astype(np.int32)
        assert oracle.energy(X, C, other) >= E


# ----------------------------------------------------------------------------------------- Lloyd
def test_lloyd_monotone_and_fixed_point():
    X, C0 = datagen.small_2d(seed=0)
    C, rho, info, tr = oracle.solve(X, C0, lloyd=True, trace=True)
    assert info["converged"] == 1
    Es = [r["E"] for r in tr]
    assert all(b <= a for a, b in zip(Es, Es[1:]))              # monotone decrease
    C_means, _ = oracle.update(X, rho, C.shape[0], C)
    np.testing.assert_array_equal(C, C_means)                   # C* = means(P*)
    rho2, _, _ = oracle.assign(X, C)
    np.testing.assert_array_equal(rho2, rho)                    # Assign(C*) = P*
    assert info["assign_passes"] == info["iters"] + 1


def test_lloyd_well_separated_recovers_component_means():
    r = np.random.default_rng(4)
    K, d, n = 6, 3, 50
    centres = np.arange(K)[:, None] * 100.0 + np.zeros((1, d))
    labels = np.repeat(np.arange(K), n)
    X = centres[labels] + 0.5 * r.normal(size=(K * n, d))
    C0 = X[np.arange(K) * n + 3]
    C, rho, info = oracle.solve(X, C0, lloyd=True)
    assert info["iters"] == 1 and info["converged"] == 1
    np.testing.assert_array_equal(rho, labels)
    for j in range(K):
        np.testing.assert_allclose(C[j], X[labels == j].mean(axis=0), rtol=1e-13)


def test_worked_example_1d_lloyd_and_aa():
    """Hand-derived trajectory on X = {0, 2, 10, 12}, C0 = {0, 2}.

    Lloyd: P^0 = (0,1,1,1) -> C^1 = (0, 8).  t=1: P^1 = (0,0,1,1) != P^0, E^1 = 0+4+4+16 = 24,
    C^2 = (1, 11).  t=2: P^2 = P^1 -> converged, E = 4, 2 iterations, 3 assignment passes.

    Algorithm 1 (m0 = 2): F^0 = C^1 - C^0 = (0, 6), G^1 = (1, 11), F^1 = G^1 - C^1 = (1, 3),
    dF_1 = (1, -3), theta = <dF,F^1>/<dF,dF> = -8/10, dG_1 = G^1 - G^0 = (1, 3),
    C^2 = G^1 - theta dG_1 = (1.8, 13.4).  t=2: assignment unchanged at an accelerated point, so
    the solver reverts to C_AU = (1, 11), which confirms: 2 iterations, 1 rejected, E = 4,
    E_trial(t=2) = 1.8^2 + 0.2^2 + 3.4^2 + 1.4^2 = 16.8.
    """
    X = np.array([[0.0], [2.0], [10.0], [12.0]])
    C0 = np.array([[0.0], [2.0]])
    C, rho, info, tr = oracle.solve(X, C0, lloyd=True, trace=True)
    np.testing.assert_array_equal(C.ravel(), [1.0, 11.0])
    np.testing.assert_array_equal(rho, [0, 0, 1, 1])
    assert (info["iters"], info["assign_passes"], info["E"]) == (2, 3, 4.0)
    assert tr[0]["E"] == 24.0
    C, rho, info, tr = oracle.solve(X, C0, trace=True)
    np.testing.assert_array_equal(C.ravel(), [1.0, 11.0])
    assert (info["iters"], info["rejected"], info["accepted"], info["E"]) == (2, 1, 0, 4.0)
    assert info["assign_passes"] == 4
    assert tr[1]["accelerated"] == 1 and tr[1]["rejected"] == 1
    assert tr[1]["E_trial"] == pytest.approx(16.8, rel=1e-14)


# ------------------------------------------------------------------------------ Algorithm 1 (AA)
@pytest.mark.parametrize("seed", range(4))
def test_aa_with_m0_is_exactly_lloyd(seed):
    X, C0 = datagen.small_2d(seed=seed)
    Cl, rl, il, tl = oracle.solve(X, C0, lloyd=True, trace=True)
    Ca, ra, ia, ta = oracle.solve(X, C0, m_max=0, trace=True)
    np.testing.assert_array_equal(Cl, Ca)
    np.testing.assert_array_equal(rl, ra)
    for f in ("iters", "assign_passes", "converged", "E"):
        assert il[f] == ia[f]
    assert ia["accepted"] == 0 and ia["rejected"] == 0
    assert [r["E"] for r in tl] == [r["E"] for r in ta]


@pytest.mark.parametrize("seed", range(4))
def test_aa_invariants(seed):
    X, C0 = datagen.small_2d(seed=seed)
    C, rho, info, tr = oracle.solve(X, C0, trace=True)
    assert info["converged"] == 1
    Es = [r["E"] for r in tr]
    assert all(b <= a for a, b in zip(Es, Es[1:]))              # stored E non-increasing
    prev = math.inf
    for r in tr:
        if r["accelerated"] and not r["rejected"]:
            assert r["E_trial"] < prev                          # accepted iterates decrease E
        prev = r["E"]
    assert info["accepted"] + info["rejected"] == sum(r["accelerated"] for r in tr)
    assert info["assign_passes"] == 1 + info["iters"] + info["rejected"]
    assert all(0 <= r["m"] <= 10 and r["m_t"] <= min(r["m"], r["t"]) for r in tr)
    C_means, _ = oracle.update(X, rho, C.shape[0], C)           # Reading R8: fixed point
    np.testing.assert_array_equal(C, C_means)
    np.testing.assert_array_equal(oracle.assign(X, C)[0], rho)
    assert info["E"] == pytest.approx(oracle.energy(X, C, rho), rel=1e-14)


def test_aa_max_iter_returns_lloyd_image():
    X, C0 = datagen.small_2d(seed=1)
    C, rho, info = oracle.solve(X, C0, max_iter=2)
    assert info["converged"] == 0 and info["iters"] == 2
    C_means, _ = oracle.update(X, rho, C.shape[0], C)
    np.testing.assert_array_equal(C, C_means)


# --------------------------------------------------------------------------- least squares, Eq. 7
@pytest.mark.parametrize("m", [1, 2, 5, 10])
def test_ls_qr_matches_svd_lstsq(m):
    r = np.random.default_rng(m)
    A = r.normal(size=(60, m))
    f = r.normal(size=60)
    theta, rank = oracle.ls_qr(A, f)
    ref = np.linalg.lstsq(A, f, rcond=None)[0]
    assert rank == m
    np.testing.assert_allclose(theta, ref, rtol=1e-10, atol=1e-12)


def test_ls_qr_truncates_dependent_columns():
    r = np.random.default_rng(7)
    A = r.normal(size=(30, 4))
    A[:, 2] = 2.0 * A[:, 0] - A[:, 1]               # third column dependent on the first two
    f = r.normal(size=30)
    theta, rank = oracle.ls_qr(A, f)
    assert rank == 2 and theta[2] == 0.0 and theta[3] == 0.0
    ref = np.linalg.lstsq(A[:, :2], f, rcond=None)[0]
    np.testing.assert_allclose(theta[:2], ref, rtol=1e-10)
    theta0, rank0 = oracle.ls_qr(np.zeros((10, 3)), r.normal(size=10))
    assert rank0 == 0 and (theta0 == 0).all()


def _with_singular_values(n, sv, seed):
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.normal(size=(n, len(sv))))
    V, _ = np.linalg.qr(r.normal(size=(len(sv), len(sv))))
    return (U * np.asarray(sv)) @ V.T


@pytest.mark.parametrize("cond", [1e6, 1e9, 1e11])
def test_ls_qr_keeps_columns_up_to_cond_1e12(cond):
    """Reading R11's cut is |R_kk| <= 1e-12 |R_00|: a history whose condition number lies between
    1e6 and 1e12 keeps every column (min |R_kk| >= sigma_min), and the QR's theta is the
    least-squares solution to the accuracy u * cond that a backward-stable solve guarantees."""
    m = 6
    A = _with_singular_values(300, np.geomspace(1.0, 1.0 / cond, m), seed=int(np.log10(cond)))
    theta_true = np.linspace(1.0, -2.0, m)
    f = A @ theta_true                               # consistent system: the exact minimiser is theta_true
    theta, rank = oracle.ls_qr(A, f)
    assert rank == m
    np.testing.assert_allclose(theta, theta_true, rtol=0, atol=1e-16 * cond * 50 * np.abs(theta_true).max())
    ref = np.linalg.lstsq(A, f, rcond=1e-14)[0]
    np.testing.assert_allclose(theta, ref, rtol=0, atol=1e-16 * cond * 50 * np.abs(theta_true).max())


def test_ls_qr_drops_a_column_dependent_to_1e_13():
    """A newest-first history whose oldest column equals a combination of the others up to 1e-13
    (relative) has |R_kk| / |R_00| far below 1e-12: that column is dropped, the rest solved."""
    r = np.random.default_rng(11)
    A = r.normal(size=(100, 4))
    A[:, 3] = A[:, 0] - 0.5 * A[:, 2] + 1e-13 * r.normal(size=100)
    f = r.normal(size=100)
    theta, rank = oracle.ls_qr(A, f)
    assert rank == 3 and theta[3] == 0.0
    np.testing.assert_allclose(theta[:3], np.linalg.lstsq(A[:, :3], f, rcond=None)[0], rtol=1e-10)
    # the same column 1e-8 away from dependence is kept at the default cut
    A[:, 3] = A[:, 0] - 0.5 * A[:, 2] + 1e-8 * r.normal(size=100)
    theta, rank = oracle.ls_qr(A, f)
    assert rank == 4


def test_ls_qr_equals_normal_equations_when_well_conditioned():
    """The LS solution through the Gram matrix and its Cholesky factor (the R of the QR)."""
    r = np.random.default_rng(8)
    A = r.normal(size=(200, 6))
    f = r.normal(size=200)
    theta, _ = oracle.ls_qr(A, f)
    L = np.linalg.cholesky(A.T @ A)
    ref = np.linalg.solve(L.T, np.linalg.solve(L, A.T @ f))
    np.testing.assert_allclose(theta, ref, rtol=1e-10)


# ------------------------------------------------------------------- Anderson on an affine map
def _contraction(n, seed, rho=0.9):
    r = np.random.default_rng(seed)
    M = r.normal(size=(n, n))
    A = rho * M / np.max(np.abs(np.linalg.eigvals(M)))
    return A, r.normal(size=n)


@pytest.mark.parametrize("n", [3, 6])
def test_aa_affine_reaches_fixed_point_in_n_plus_1_steps(n):
    A, b = _contraction(n, seed=n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    traj = oracle.aa_affine(A, b, np.zeros(n), m=n, iters=n + 2, rank_tol=1e-14)
    err = np.linalg.norm(traj[n + 1] - xstar) / np.linalg.norm(xstar)
    assert err < 1e-9
    # the same number of plain fixed-point steps is still far from x*
    x = np.zeros(n)
    for _ in range(n + 1):
        x = A @ x + b
    assert np.linalg.norm(x - xstar) / np.linalg.norm(xstar) > 1e-3


def test_aa_affine_m0_is_picard_iteration():
    A, b = _contraction(4, seed=11)
    traj = oracle.aa_affine(A, b, np.ones(4), m=0, iters=5)
    x = np.ones(4)
    for k in range(5):
        x = A @ x + b
        np.testing.assert_allclose(traj[k + 1], x, rtol=1e-14)


def test_aa_affine_first_step_closed_form():
    """m=1 after two Picard steps: theta = <dF,f1>/<dF,dF>, x2 = g1 - theta (g1 - g0)."""
    A, b = _contraction(3, seed=5)
    x0 = np.zeros(3)
    g0 = A @ x0 + b
    f0 = g0 - x0
    x1 = g0
    g1 = A @ x1 + b
    f1 = g1 - x1
    dF = f1 - f0
    th = dF @ f1 / (dF @ dF)
    x2 = g1 - th * (g1 - g0)
    traj = oracle.aa_affine(A, b, x0, m=1, iters=2)
    np.testing.assert_allclose(traj[2], x2, rtol=1e-13)


# --------------------------------------------------------------------------------- dynamic m rule
def test_m_rule_scripted():
    # t <= 2: never adjusted (Reading R4)
    assert oracle.m_rule(2, 10, 1, 5.0, np.inf, np.inf) == 2
    assert oracle.m_rule(2, 10, 2, 5.0, 6.0, np.inf) == 2
    # energy went up (num < 0 < eps1*den): decrease
    assert oracle.m_rule(3, 10, 5, 10.5, 10.0, 11.0) == 2
    # small decrease: ratio 0.01 < 0.02 -> decrease; clamps at 0
    assert oracle.m_rule(3, 10, 5, 9.99, 10.0, 11.0) == 2
    assert oracle.m_rule(0, 10, 5, 9.99, 10.0, 11.0) == 0
    # large decrease: ratio 0.6 > 0.5 -> increase; clamps at m_max
    assert oracle.m_rule(3, 10, 5, 9.4, 10.0, 11.0) == 4
    assert oracle.m_rule(10, 10, 5, 9.4, 10.0, 11.0) == 10
    # in between: unchanged (ratio 0.3)
    assert oracle.m_rule(3, 10, 5, 9.7, 10.0, 11.0) == 3
    # boundaries: ratio exactly eps1 / eps2 leaves m unchanged
    # (exactly representable: den = 1, num = 0.25 and 0.5)
    assert oracle.m_rule(3, 10, 5, 0.75, 1.0, 2.0, eps1=0.25) == 3
    assert oracle.m_rule(3, 10, 5, 0.5, 1.0, 2.0, eps2=0.5) == 3
    assert oracle.m_rule(3, 10, 5, 0.4375, 1.0, 2.0, eps2=0.5) == 4
    # den = 0 (Reading R5): num > 0 -> increase, num < 0 -> decrease, num = 0 -> unchanged
    assert oracle.m_rule(3, 10, 5, 9.0, 10.0, 10.0) == 4
    assert oracle.m_rule(3, 10, 5, 11.0, 10.0, 10.0) == 2
    assert oracle.m_rule(3, 10, 5, 10.0, 10.0, 10.0) == 3


# --------------------------------------------- fixed m (Section 3, "Settings of m"; Tab. 2)
@pytest.mark.parametrize("seed", range(3))
def test_fixed_m0_is_exactly_lloyd(seed):
    # m held at 0 never mixes: the Lloyd map, pass for pass (while the dynamic rule started at
    # m = 0 does raise m on these data, so the flag is what keeps it at 0)
    X, C0 = datagen.small_2d(seed=seed)
    Cl, rl, il = oracle.solve(X, C0, lloyd=True)
    Cf, rf, jf = oracle.solve(X, C0, m_init=0, fixed_m=1)
    np.testing.assert_array_equal(Cl, Cf)
    np.testing.assert_array_equal(rl, rf)
    for f in ("iters", "assign_passes", "converged", "E"):
        assert il[f] == jf[f]
    assert jf["accepted"] == 0 and jf["rejected"] == 0
    _, _, _, tr = oracle.solve(X, C0, m_init=0, trace=True)
    assert max(r["m"] for r in tr) > 0


@pytest.mark.parametrize("m", [2, 5])
@pytest.mark.parametrize("seed", range(3))
def test_fixed_m_keeps_m_and_invariants(seed, m):
    X, C0 = datagen.small_2d(seed=seed)
    C, rho, info, tr = oracle.solve(X, C0, m_init=m, m_max=10, fixed_m=1, trace=True)
    assert info["converged"] == 1 and info["m_final"] == m
    assert all(r["m"] == m for r in tr)
    assert all(math.isnan(r["margin_lo"]) and math.isnan(r["margin_hi"]) for r in tr)
    assert all(r["m_t"] <= min(m, r["t"]) for r in tr)
    Es = [r["E"] for r in tr]
    assert all(b <= a for a, b in zip(Es, Es[1:]))              # stored E non-increasing
    prev = math.inf
    for r in tr:
        if r["accelerated"] and not r["rejected"]:
            assert r["E_trial"] < prev                          # accepted iterates decrease E
        prev = r["E"]
    assert info["assign_passes"] == 1 + info["iters"] + info["rejected"]
    C_means, _ = oracle.update(X, rho, C.shape[0], C)           # Reading R8: fixed point
    np.testing.assert_array_equal(C, C_means)
    np.testing.assert_array_equal(oracle.assign(X, C)[0], rho)


def test_fixed_m_is_clamped_to_m_max():
    X, C0 = datagen.small_2d(seed=0)
    Ca, ra, ia = oracle.solve(X, C0, m_init=7, m_max=3, fixed_m=1)
    Cb, rb, ib = oracle.solve(X, C0, m_init=3, m_max=3, fixed_m=1)
    np.testing.assert_array_equal(Ca, Cb)
    assert ia["iters"] == ib["iters"] and ia["m_final"] == 3


# --------------------------------------------------------------- K-Means++ seeding (D^2 sampling)
def test_kmeanspp_first_pick_is_uniform_index():
    X = np.arange(10, dtype=np.float64).reshape(10, 1)
    for u0, want in ((0.0, 0), (0.05, 0), (0.1, 1), (0.55, 5), (0.999, 9)):
        idx, C = oracle.kmeanspp(X, 1, [u0])
        assert idx[0] == want and C[0, 0] == want


def test_kmeanspp_inverse_cdf_by_hand():
    # points 0, 1, 3, 6 on a line; first centre x = 0 -> weights 0, 1, 9, 36 (W = 46):
    # u W in (0, 1] -> x = 1, (1, 10] -> x = 3, (10, 46) -> x = 6
    X = np.array([[0.0], [1.0], [3.0], [6.0]])
    for uW, want in ((0.5, 1), (0.99, 1), (1.5, 2), (5.0, 2), (9.9, 2), (10.5, 3), (20.0, 3), (45.9, 3)):
        idx, _ = oracle.kmeanspp(X, 2, [0.0, uW / 46.0])
        assert idx[1] == want, (uW, idx)
    # third pick with centres {0, 6}: weights 0, min(1, 25) = 1, min(9, 9) = 9, 0 (W = 10)
    for uW, want in ((0.5, 1), (2.0, 2), (9.9, 2)):
        idx, _ = oracle.kmeanspp(X, 3, [0.0, 20.0 / 46.0, uW / 10.0])
        assert list(idx) == [0, 3, want], (uW, idx)


def test_kmeanspp_never_repeats_and_n_equals_k_is_a_permutation():
    r = np.random.default_rng(3)
    X = r.normal(size=(12, 2))
    for s in range(5):
        idx, C = oracle.kmeanspp(X, 12, np.random.default_rng(s).random(12))
        assert sorted(idx) == list(range(12))
        np.testing.assert_array_equal(C, X[idx])
    # duplicates of a chosen point have weight 0 and are never drawn
    Xd = np.vstack([X[:4], X[:4], X[:4]])
    idx, _ = oracle.kmeanspp(Xd, 4, [0.0, 0.3, 0.6, 0.9])
    assert len({tuple(Xd[i]) for i in idx}) == 4


def test_kmeanspp_all_identical_falls_back_to_uniform():
    X = np.ones((8, 3))
    idx, _ = oracle.kmeanspp(X, 3, [0.0, 0.5, 0.99])
    assert list(idx) == [0, 4, 7]


def test_kmeanspp_one_pick_per_separated_cluster():
    # 10 tight clusters 100 apart: after a pick, the other clusters carry all but ~1e-8 of the
    # weight, so D^2 sampling picks one sample from each
    r = np.random.default_rng(5)
    centres = 100.0 * np.arange(10)[:, None] * np.array([[1.0, 0.5]])
    lab = r.integers(0, 10, size=5000)
    X = centres[lab] + 0.01 * r.normal(size=(5000, 2))
    for s in range(5):
        idx, _ = oracle.kmeanspp(X, 10, np.random.default_rng(100 + s).random(10))
        assert sorted(lab[idx]) == list(range(10))


# ------------------------------------------------------------------------------ one loop pass
def test_step_reproduces_solve_pass_by_pass():
    """``step`` is the body of ``solve``: driving it from Algorithm 1's first line gives the same
    trace records, counts and result bit for bit (the step-parity tests start the GPU and the
    oracle from one exported state through it)."""
    X, C0 = datagen.small_2d(seed=1)
    C_ref, rho_ref, info_ref, tr_ref = oracle.solve(X, C0, trace=True)
    rho0, _, _ = oracle.assign(X, C0)
    G, _ = oracle.update(X, rho0, C0.shape[0], C0)
    st = dict(C=G.copy(), CAU=G.copy(), F=G - C0, count=0, Pprev=rho0, t=1, m=2, from_lloyd=1,
              E_prev=math.inf, E_prev2=math.inf, assign_passes=1)
    recs = []
    while not st.get("done") and st["t"] <= 1000:
        st, rec = oracle.step(X, st)
        recs.append(rec)
    assert [r["E"] for r in recs] == [r["E"] for r in tr_ref]
    assert [(r["m"], r["rank"], r["rejected"]) for r in recs] == [(r["m"], r["rank"], r["rejected"]) for r in tr_ref]
    assert (st["t"], st["accepted"], st["rejected"], st["assign_passes"]) == (
        info_ref["iters"], info_ref["accepted"], info_ref["rejected"], info_ref["assign_passes"])
    np.testing.assert_array_equal(st["C"], C_ref)
    np.testing.assert_array_equal(st["Pprev"], rho_ref)
    assert st["E"] == info_ref["E"]
