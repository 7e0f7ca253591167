"""kmeans_update_static: the update step without any device allocation.

Some callers cannot allocate device memory (an allocator of their own that must not re-enter
cudaMalloc, programs that allocate everything at start-up).  This file is collected last so that
a run stopping at the first failure has already run every other test.  It calls the entry point
through the C ABI with preallocated outputs and checks:
* that the calls allocate nothing: the device's free memory (cudaMemGetInfo) and torch's
  allocated and reserved bytes are the same before and after two calls in a row;
* its output against the FP64 oracle's update (Eq. 4) and against kmeans_update, bit for bit
  (same block count, same order of the partial sums), on two calls in a row (the shared scratch
  array keeps the previous call's contents);
* the shape limit: the largest K the shared-memory bins accept at d = 16 in FP64 works and
  matches kmeans_update, the next K is rejected by both.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1805_10638_gb300 as km
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


def _data(N, d, K, dtype, seed):
    r = np.random.default_rng(seed)
    X = (r.normal(size=(N, d)) * 10 + 50).astype(dtype)
    rho = r.integers(0, K - 1, size=N).astype(np.int32)          # last cluster empty
    Cp = r.normal(size=(K, d)).astype(dtype)
    return X, rho, Cp


def _memory():
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_allocated(), torch.cuda.memory_reserved()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_update_static_allocates_nothing_and_matches(dtype):
    need_gpu()
    ctx = km.Context(0)
    shapes = [(200_003, 3, 256), (50_000, 16, 40)]
    inputs = []
    for call, (N, d, K) in enumerate(shapes):
        X, rho, Cp = _data(N, d, K, dtype, seed=call + 17)
        dev = [torch.from_numpy(a).cuda() for a in (X, rho, Cp)]
        outs = (torch.empty_like(dev[2]), torch.empty(K, dtype=torch.int64, device="cuda"))
        ref = km.kmeans_update(ctx, *dev[:2], K, dev[2])
        inputs.append((X, rho, Cp, K, dev, outs, ref))
    # a first call per shape, then the measured calls: kernels load lazily (into a code pool that
    # grows in 2 MiB steps), torch's fill kernels used below included
    for X, rho, Cp, K, dev, outs, ref in inputs:
        outs[0].fill_(-1)
        outs[1].fill_(-1)
        km.kmeans_update_static(dev[0], dev[1], K, dev[2], C_out=outs[0], counts=outs[1])
    before = _memory()
    for X, rho, Cp, K, dev, outs, ref in inputs:                     # two calls in a row
        outs[0].fill_(-1)
        outs[1].fill_(-1)
        km.kmeans_update_static(dev[0], dev[1], K, dev[2], C_out=outs[0], counts=outs[1])
    after = _memory()
    assert after == before, (before, after)
    for X, rho, Cp, K, dev, outs, ref in inputs:
        C_s, n_s = outs[0].cpu().numpy(), outs[1].cpu().numpy()
        np.testing.assert_array_equal(C_s, ref[0].cpu().numpy())     # bitwise: same partials, same order
        np.testing.assert_array_equal(n_s, ref[1].cpu().numpy())
        C_o, n_o = oracle.update(X, rho, K, Cp)
        np.testing.assert_array_equal(n_s, n_o)
        assert rel_err(C_s, C_o) < (1e-13 if dtype == np.float64 else 1e-6)
        assert np.array_equal(C_s[-1], Cp[-1])                        # empty cluster keeps C_prev
    ctx.close()


def test_update_static_shape_limit_matches_update():
    """Largest K accepted at d = 16 in FP64 (the pass kernel's shared memory binds first): same
    result as kmeans_update; K + 1 is rejected by both with KM_EINVAL."""
    need_gpu()
    L = km.load()
    d, N = 16, 4_000

    def status(K):
        X = torch.zeros((N, d), dtype=torch.float64, device="cuda")
        rho = torch.zeros(N, dtype=torch.int32, device="cuda")
        C = torch.zeros((K, d), dtype=torch.float64, device="cuda")
        out = torch.empty_like(C)
        data = km._lib.make_data(X)
        s = L.kmeans_update_static(ctypes.byref(data), rho.data_ptr(), K, C.data_ptr(), out.data_ptr(), None, None)
        torch.cuda.synchronize()
        return s

    lo, hi = 1, 2048
    assert status(lo) == 0 and status(hi) == 1
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if status(mid) == 0:
            lo = mid
        else:
            hi = mid
    Kmax = lo
    assert Kmax == 168                                    # the limit the header states
    ctx = km.Context(0)
    X, rho, Cp = _data(N, d, Kmax, np.float64, seed=5)
    dev = [torch.from_numpy(a).cuda() for a in (X, rho, Cp)]
    C_s, n_s = km.kmeans_update_static(dev[0], dev[1], Kmax, dev[2])
    C_r, n_r = km.kmeans_update(ctx, dev[0], dev[1], Kmax, dev[2])
    np.testing.assert_array_equal(C_s.cpu().numpy(), C_r.cpu().numpy())
    np.testing.assert_array_equal(n_s.cpu().numpy(), n_r.cpu().numpy())
    C2 = torch.zeros((Kmax + 1, d), dtype=torch.float64, device="cuda")
    with pytest.raises(km.KmeansError) as e:
        km.kmeans_update(ctx, dev[0], dev[1], Kmax + 1, C2)
    assert e.value.status == 1
    ctx.close()


def test_update_static_rejects_oversized():
    need_gpu()
    X = torch.zeros((10, 20), dtype=torch.float32, device="cuda")     # d > 16
    with pytest.raises(km.KmeansError):
        km.kmeans_update_static(X, torch.zeros(10, dtype=torch.int32, device="cuda"), 2,
                                torch.zeros((2, 20), dtype=torch.float32, device="cuda"))
