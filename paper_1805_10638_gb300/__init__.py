"""GB300 (sm_103a) K-Means with Anderson acceleration.

The compute path is the CUDA library ``libkmeans_aa.so`` (C ABI in ``include/kmeans_aa.h``);
this package is its thin ctypes binding.  See ``_lib`` for the calls.
"""
from ._lib import (KM_BF16_F32, KM_F32, KM_F64, Context, KmeansError, Server, batch_describe,  # noqa: F401
                   default_params, kmeans_assign, kmeans_energy, kmeans_lsq, kmeans_seed_pp, kmeans_solve,
                   kmeans_solve_batched, kmeans_solve_host, kmeans_solve_passes, kmeans_update, kmeans_update_static,
                   load)
