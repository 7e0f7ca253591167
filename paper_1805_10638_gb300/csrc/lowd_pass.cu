// Low-dimensional assignment pass (d = 1..16) for sm_103a.
//
// One launch = one pass over X that computes, per sample, the assignment step (Eq. 3), and
// fuses the O(N) work of the same pass:
//   - the residual r_i = x_i - c_{rho_i} in the direct form, its squared norm (the energy term
//     of Eq. 1) and per-cluster residual sums and counts (the update step, Eq. 4, written
//     relative to the current centroids so that F = G(C) - C comes out without cancellation);
//   - the number of samples whose assignment changed (the convergence test of Algorithm 1);
//   - in the last block to finish, the fixed-order reduction of the per-block partials and the
//     head of Algorithm 1 (convergence test, dynamic m, energy safeguard).
//
// FP32 path: distances as ||c'||^2 - 2 x'.c' with x' = x - o, c' = c - o (o = an origin near
// the data), D FMAs per (sample, centroid) pair on CUDA cores, packed two samples per
// fma.rn.f32x2.  The argmin over K runs in chunks of 8 (or 16) centroids: a 3-input min tree gives the
// chunk minimum, and only the best chunk index, the best value and the second-best chunk
// minimum are tracked.  After the scan the best chunk is re-scored (bit-identical arithmetic)
// to find the lowest index attaining the minimum and the second-best value.  If the top-2 gap
// is within twice the rounding-error bound of the expansion the row is re-scored over all K in
// the direct form sum (x - c)^2 (lowest index wins exact ties).
//
// FP64 path: direct form sum (x - c)^2 with explicitly rounded operations (no contraction),
// ascending j with strict '<', i.e. the same arithmetic as the FP64 oracle.
//
// Determinism: per-cluster sums go to per-warp shared-memory bins; within a warp, lanes with the
// same label are combined by the lowest such lane in lane order (__match_any_sync); warps are
// combined in warp order and blocks in block order.  FP32 solver passes with d <= FX_MAX_D sum in
// 64-bit fixed point instead (shared-memory, then global integer atomics into per-solve totals),
// which is exact and so independent of the order.  No floating-point atomics.
#include "lowd_pass.cuh"
#include "lowd_inst.cuh"

namespace km {

namespace {

// Block b of `gridDim.x` takes the half distances of its share of the centroids (hprep_body).
__global__ void __launch_bounds__(1024) k_hprep(PassArgs a, int mode)
{
    __shared__ float s_r[3 * 32];
    hprep_dispatch(a, mode, s_r, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024) k_hprep_batch(BatchPass b)
{
    __shared__ float s_r[3 * 32];
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const PassArgs& a = b.args[b.items[it].x];
        if (a.ham) hprep_dispatch(a, b.mode, s_r);
        __syncthreads();
    }
}

// Groups of the group bounds, once per solve from C^0: the centroids sorted by the Morton code of
// their coordinates (each dimension scaled to the bounding box and cut to 30/d bits, ties by index;
// bitonic sort of (code, index) pairs in shared memory) and cut into hg runs of consecutive ones,
// so that a group holds nearby centroids.  Any grouping gives valid bounds; nearby centroids give
// tighter ones.  One block.
__global__ void __launch_bounds__(1024) k_groups(const double* C, int K, int d, int hg, int* perm, int* goff)
{
    extern __shared__ unsigned long long s_key[];   // [P] (code << 32 | index)
    __shared__ double s_lo[16], s_hi[16];
    const int tid = threadIdx.x;
    int P = 1;
    while (P < K) P <<= 1;
    if (tid < d) {
        double lo = C[tid], hi = C[tid];
        for (int j = 1; j < K; ++j) {
            lo = fmin(lo, C[(size_t)j * d + tid]);
            hi = fmax(hi, C[(size_t)j * d + tid]);
        }
        s_lo[tid] = lo;
        s_hi[tid] = hi;
    }
    __syncthreads();
    const int B = d >= 30 ? 1 : 30 / d;
    for (int j = tid; j < P; j += blockDim.x) {
        unsigned long long key = ~0ull;
        if (j < K) {
            unsigned code = 0;
            for (int k = 0; k < d; ++k) {
                const double w = s_hi[k] - s_lo[k];
                double f = w > 0.0 ? (C[(size_t)j * d + k] - s_lo[k]) / w : 0.0;
                unsigned q = (unsigned)(f * (double)(1u << B));
                q = q > (1u << B) - 1u ? (1u << B) - 1u : q;
                for (int b = 0; b < B; ++b) code |= ((q >> b) & 1u) << (b * d + k);
            }
            key = ((unsigned long long)code << 32) | (unsigned)j;
        }
        s_key[j] = key;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P; i += blockDim.x) {
                const int partner = i ^ stride;
                if (partner > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long x = s_key[i], y = s_key[partner];
                    if ((x > y) == up) {
                        s_key[i] = y;
                        s_key[partner] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int p = tid; p < K; p += blockDim.x) perm[p] = (int)(s_key[p] & 0xffffffffu);
    for (int gi = tid; gi <= hg; gi += blockDim.x) goff[gi] = (int)((long long)K * gi / hg);
}

}  // namespace

cudaError_t launch_groups(const double* C, int K, int d, int hg, int* perm, int* goff, cudaStream_t s)
{
    int P = 1;
    while (P < K) P <<= 1;
    const size_t smem = (size_t)P * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_groups<<<1, 1024, smem, s>>>(C, K, d, hg, perm, goff);
    return cudaGetLastError();
}

cudaError_t launch_hprep(const PassArgs& a, int mode, cudaStream_t s)
{
    const int parts = a.K / 32 < 1 ? 1 : (a.K / 32 > 16 ? 16 : a.K / 32);   // >= 32 centroids per block
    k_hprep<<<parts, 1024, 0, s>>>(a, mode);
    return cudaGetLastError();
}

cudaError_t launch_hprep_batch(const BatchPass& b, int grid, cudaStream_t s)
{
    k_hprep_batch<<<grid, 1024, 0, s>>>(b);
    return cudaGetLastError();
}

int pass_lowd_dp(int d)
{
    return ((2 * (d + 1) + 3) / 4 * 4) / 2;
}

size_t pass_lowd_smem(int prec, int d, int K, int Kpad, bool bins, int hq_cap, int hg)
{
    // the fixed-point layout of the solver's TRIAL / REVERT passes is never larger than the per-warp one
    return layout(prec != KM_F64, d, pass_lowd_dp(d), K, Kpad, bins, hq_cap, false, hg).total;
}

cudaError_t launch_pass_lowd(const PassArgs& a, int prec, int d, int nb, cudaStream_t s)
{
    const size_t smem = pass_lowd_smem(prec, d, a.K, a.Kpad, (a.flags & F_BINS) != 0, a.ham ? a.hq_cap : 0,
                                       a.ham ? a.hg : 0);
    if (prec == KM_F64) return lowd_launch_f64(a, d, nb, smem, s);
    // FP32 passes without update bins and bounds: the assignment-only kernel
    if (!(a.flags & F_BINS) && !a.ham) return lowd_launch_f32_ao(a, d, nb, smem, s);
    return lowd_launch_f32(a, d, nb, smem, s);
}

cudaError_t launch_pass_lowd_batch(const BatchPass& b, int prec, int d, int grid, size_t smem, cudaStream_t s,
                                   int variant)
{
    if (prec == KM_F64) return lowd_batch_launch_f64(b, d, grid, smem, s);
    return variant == 1 ? lowd_batch_launch_f32_v1(b, d, grid, smem, s) : lowd_batch_launch_f32(b, d, grid, smem, s);
}

int pass_lowd_occupancy_ao(int d, size_t smem) { return lowd_occupancy_f32_ao(d, smem); }

int pass_lowd_occupancy(int prec, int d, size_t smem)
{
    return prec == KM_F64 ? lowd_occupancy_f64(d, smem) : lowd_occupancy_f32(d, smem);
}

int pass_lowd_batch_occupancy(int prec, int d, size_t smem, int variant)
{
    if (prec == KM_F64) return lowd_batch_occupancy_f64(d, smem);
    return variant == 1 ? lowd_batch_occupancy_f32_v1(d, smem) : lowd_batch_occupancy_f32(d, smem);
}

}  // namespace km
