"""kmeans_update_static: the update step without any device allocation.

Some callers cannot allocate device memory (an allocator of their own that must not re-enter
cudaMalloc, programs that allocate everything at start-up).  This file is collected last so that
a run stopping at the first failure has already run every other test.  It calls the entry point
through the C ABI and checks it against kmeans_update on the same inputs, twice in a row (the
shared scratch array keeps the previous call's contents).
"""
import numpy as np
import pytest
import torch

import paper_1805_10638_gb300 as km
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_update_static_matches_update_twice(dtype):
    need_gpu()
    ctx = km.Context(0)
    for call, (N, d, K) in enumerate([(200_003, 3, 256), (50_000, 16, 40)]):
        r = np.random.default_rng(call + 17)
        X = (r.normal(size=(N, d)) * 10 + 50).astype(dtype)
        rho = r.integers(0, K - 1, size=N).astype(np.int32)          # last cluster empty
        Cp = r.normal(size=(K, d)).astype(dtype)
        Xd, rd, Cd = (torch.from_numpy(a).cuda() for a in (X, rho, Cp))
        C_ref, n_ref = km.kmeans_update(ctx, Xd, rd, K, Cd)
        C_s, n_s = km.kmeans_update_static(Xd, rd, K, Cd)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(n_s.cpu().numpy(), n_ref.cpu().numpy())
        tol = 1e-13 if dtype == np.float64 else 1e-6
        assert rel_err(C_s.cpu().numpy(), C_ref.cpu().numpy()) < tol
    ctx.close()


def test_update_static_rejects_oversized():
    need_gpu()
    X = torch.zeros((10, 20), dtype=torch.float32, device="cuda")     # d > 16
    with pytest.raises(km.KmeansError):
        km.kmeans_update_static(X, torch.zeros(10, dtype=torch.int32, device="cuda"), 2,
                                torch.zeros((2, 20), dtype=torch.float32, device="cuda"))
