"""Serving (kmeans_server_*) through the C ABI: admission against an HBM budget, continuous
batching of low-d requests, large requests on a second stream.

The bar: every request's result in the mix is the same as the same request solved alone with
kmeans_solve_host, to the bit (the same kernels run with the same per-request decomposition),
and the budget is never exceeded."""
import numpy as np
import pytest
import torch

import datagen
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _requests(n_small=20, n_large=2, seed=0):
    r = np.random.default_rng(seed)
    reqs = []
    for i in range(n_small):
        d = int(r.choice([2, 3, 16]))
        N = int(np.exp(r.uniform(np.log(500), np.log(30000))))
        K = int(np.exp(r.uniform(np.log(4), np.log(48))))
        dt = np.float64 if i % 4 == 0 else np.float32
        X, C0 = datagen.batched_instance(N, d, K, 7000 + i, dtype=dt)
        p = dict(lloyd_only=1) if i % 3 == 0 else dict(m_max=10)
        reqs.append(dict(X=_pinned(X), C0=_pinned(C0), Xb=None, p=p))
    for j in range(n_large):
        X, C0 = datagen.batched_instance(20000, 32, 64, 9000 + j, dtype=np.float32)
        reqs.append(dict(X=_pinned(X), C0=_pinned(C0), Xb=_pinned(datagen.to_bf16_bits(X).view(np.int16)),
                         p=dict(m_max=10)))
    order = r.permutation(len(reqs))
    return [reqs[i] for i in order]


def _alone(reqs):
    ctx = km.Context(0)
    out = []
    for q in reqs:
        Xb = q["Xb"].view(torch.bfloat16) if q["Xb"] is not None else None
        C, rho, info = km.kmeans_solve_host(ctx, q["X"], q["C0"], X_bf16=Xb, **q["p"])
        out.append((C.clone(), rho.clone(), info))
    return out


def test_serving_mix_equals_alone():
    need_gpu()
    reqs = _requests()
    budget = 48 << 20
    srv = km.Server(0, hbm_budget=budget, max_slots=6, max_large=1)
    tickets, results = [], {}
    saw_waiting = False
    pending = list(range(len(reqs)))
    steps = 0
    while len(results) < len(reqs):
        # a few arrivals every other step
        if pending and steps % 2 == 0:
            for _ in range(3):
                if pending:
                    i = pending.pop(0)
                    q = reqs[i]
                    Xb = q["Xb"].view(torch.bfloat16) if q["Xb"] is not None else None
                    tickets.append((i, srv.submit(q["X"], q["C0"], X_bf16=Xb, **q["p"])))
        srv.step()
        st = srv.stats()
        saw_waiting |= st["waiting"] > 0
        assert st["pool_used"] <= budget and st["pool_peak"] <= budget
        for i, t in tickets:
            if i not in results:
                res = srv.poll(t)
                if res is not None:
                    results[i] = res
        steps += 1
        assert steps < 200000
    assert saw_waiting, "the budget and slot limits never made a request wait"
    alone = _alone(reqs)
    for i, (C, rho, info) in results.items():
        Ca, ra, ia = alone[i]
        assert C.numpy().tobytes() == Ca.numpy().tobytes(), f"request {i}: centroids differ"
        assert np.array_equal(rho.numpy(), ra.numpy()), f"request {i}: assignments differ"
        for f in ("iters", "accepted", "rejected", "assign_passes", "converged", "E", "status"):
            assert info[f] == ia[f], f"request {i}: {f} {info[f]} != {ia[f]}"
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pool_used"] == 0
    srv.close()


def test_serving_rejects_oversized_and_idles():
    need_gpu()
    srv = km.Server(0, hbm_budget=1 << 20, max_slots=2, max_large=0)
    X, C0 = datagen.batched_instance(200000, 3, 16, 1, dtype=np.float32)
    with pytest.raises(km.KmeansError):
        srv.submit(_pinned(X), _pinned(C0))
    assert srv.step() == 0
    X = torch.randn(100, 32).pin_memory()
    with pytest.raises(km.KmeansError):          # d > 16 needs BF16 and a large lane
        srv.submit(X, X[:4].clone().pin_memory())
    srv.close()


def test_served_results_match_the_fp64_oracle():
    """Every served request (FP64 and FP32 low-d in the continuous batch, a BF16 request on a large
    lane; Lloyd and Algorithm 1) against the FP64 oracle: the returned (C, P, E) is exact arithmetic
    on its own assignment (E to 1e-6, C = the means of P to 1e-6, P the argmin at C off the tie
    band), and its final energy equals the oracle's own solve from the same C0 to 1e-6 relative."""
    need_gpu()
    import oracle
    from gpu_util import check_assignment, rel_err
    reqs = _requests(n_small=12, n_large=1, seed=3)
    srv = km.Server(0, hbm_budget=256 << 20, max_slots=4, max_large=1)
    tickets = []
    for i, q in enumerate(reqs):
        Xb = q["Xb"].view(torch.bfloat16) if q["Xb"] is not None else None
        tickets.append((i, srv.submit(q["X"], q["C0"], X_bf16=Xb, **q["p"])))
    results = {}
    steps = 0
    while len(results) < len(reqs):
        srv.step()
        for i, t in tickets:
            if i not in results:
                res = srv.poll(t)
                if res is not None:
                    results[i] = res
        steps += 1
        assert steps < 200000
    srv.close()
    for i, (C, rho, info) in results.items():
        q = reqs[i]
        X = q["X"].numpy()
        C, rho = C.numpy(), rho.numpy()
        assert info["converged"] == 1 and info["status"] == 0, (i, info)
        E_at = oracle.energy(X, C, rho)
        assert abs(info["E"] - E_at) <= 1e-6 * E_at, (i, info["E"], E_at)
        Cm, _ = oracle.update(X, rho, C.shape[0], C)
        assert rel_err(C, Cm) <= 1e-6, i
        check_assignment(X, C, rho, f"request {i}")
        lloyd = q["p"].get("lloyd_only", 0) == 1
        Co, ro, io = oracle.solve(X, q["C0"].numpy(), lloyd=lloyd, m_max=10)
        assert abs(info["E"] - io["E"]) <= 1e-6 * io["E"], (i, info, io)
        if X.dtype == np.float64:
            assert (info["iters"], info["accepted"], info["rejected"]) == (io["iters"], io["accepted"], io["rejected"])
