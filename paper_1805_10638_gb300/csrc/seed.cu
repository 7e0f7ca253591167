// K-Means++ seeding on the device (sm_103a): the D^2 weighting of Arthur and Vassilvitskii, the
// initialiser the paper names beside random seeding (Sections 1 and 3).  The uniforms are the
// caller's (one per chosen row), so a seeding is reproducible and can be checked row for row.
//
// k_pp_weights : one pass over X per chosen row.  Each row's weight w_i, the squared distance to
//                its nearest chosen row, takes the minimum with the distance to the newest one,
//                in FP64 with the rounding of a plain sequential loop (separately rounded
//                multiplies and adds, no fused multiply-add).  Blocks own contiguous row ranges and
//                write their weight sums (fixed-order reduction).
// k_pp_pick    : one block turns the uniform u into a row by inverse-CDF sampling in index order:
//                a fixed-order scan of the block sums finds the block whose range holds u W, and a
//                scan of that block's rows finds the first row whose running sum exceeds u W.  If
//                rounding leaves no such row, the last row of that block with w > 0 is taken; if
//                W = 0 (fewer distinct rows than chosen ones) the row is floor(u N).

#include "runtime.cuh"

#include <climits>

namespace km {
namespace {

constexpr int PP_THREADS = 256;
constexpr int PICK_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(PP_THREADS) k_pp_weights(const T* __restrict__ X, int64_t N, int d,
                                                          const T* C, int c, int64_t R, double* w, double* P)
{
    const int64_t lo = (int64_t)blockIdx.x * R;
    const int64_t hi = lo + R < N ? lo + R : N;
    const T* cp = C + (size_t)(c - 1) * d;            // the newest chosen row
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            const double t = __dsub_rn((double)X[(size_t)i * d + k], (double)cp[k]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        double wi = c == 1 ? s : w[i];
        if (c > 1 && s < wi) wi = s;
        w[i] = wi;
        acc = __dadd_rn(acc, wi);
    }
    __shared__ double red[PP_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < PP_THREADS / 32; ++k) s = __dadd_rn(s, red[k]);
        P[blockIdx.x] = s;
    }
}

// Inclusive scan of one value per thread (Hillis-Steele, fixed order); returns the thread's
// exclusive prefix; *total gets the sum.
__device__ double block_exclusive_scan(double v, double* buf, double* total)
{
    const int t = threadIdx.x;
    buf[t] = v;
    __syncthreads();
    for (int off = 1; off < PICK_THREADS; off <<= 1) {
        const double add = t >= off ? buf[t - off] : 0.0;
        __syncthreads();
        if (t >= off) buf[t] = __dadd_rn(buf[t], add);
        __syncthreads();
    }
    const double ex = t > 0 ? buf[t - 1] : 0.0;
    *total = buf[PICK_THREADS - 1];
    __syncthreads();
    return ex;
}

__device__ __forceinline__ int64_t uniform_row(double u, int64_t N)
{
    int64_t i = (int64_t)floor(__dmul_rn(u, (double)N));
    return i > N - 1 ? N - 1 : (i < 0 ? 0 : i);
}

template <typename T>
__global__ void __launch_bounds__(PICK_THREADS) k_pp_pick(const T* __restrict__ X, int64_t N, int d, T* C,
                                                         int32_t* idx, const double* u, int c, const double* w,
                                                         const double* P, int NB, int64_t R)
{
    __shared__ double buf[PICK_THREADS];
    __shared__ long long s_pick, s_last;
    __shared__ int s_blk, s_blast;
    __shared__ double s_base;
    const int t = threadIdx.x;
    const double uc = u[c];
    if (t == 0) {
        s_pick = LLONG_MAX;
        s_last = -1;
        s_blk = INT_MAX;
        s_blast = -1;
    }
    __syncthreads();
    int64_t pick = -1;
    if (c == 0) {
        pick = uniform_row(uc, N);
    } else {
        // blocks: thread t owns the block sums [t q, (t+1) q)
        const int q = (NB + PICK_THREADS - 1) / PICK_THREADS;
        const int b0 = t * q, b1 = b0 + q < NB ? b0 + q : NB;
        double loc = 0.0;
        for (int b = b0; b < b1; ++b) loc = __dadd_rn(loc, P[b]);
        double W;
        const double ex = block_exclusive_scan(loc, buf, &W);
        if (!(W > 0.0)) {
            pick = uniform_row(uc, N);
        } else {
            const double target = __dmul_rn(uc, W);
            double run = ex;
            for (int b = b0; b < b1; ++b) {
                const double nxt = __dadd_rn(run, P[b]);
                if (P[b] > 0.0) {
                    atomicMax(&s_blast, b);
                    if (nxt > target) {
                        atomicMin(&s_blk, b);
                        break;
                    }
                }
                run = nxt;
            }
            __syncthreads();
            // the first block whose running sum passes the target (else the last block with weight);
            // its owner recomputes the running sum in front of it
            int blk = s_blk;
            const bool found = blk != INT_MAX;
            if (!found) blk = s_blast;
            __syncthreads();
            if (blk >= b0 && blk < b1) {
                double r2 = ex;
                for (int b = b0; b < blk; ++b) r2 = __dadd_rn(r2, P[b]);
                s_base = r2;
            }
            __syncthreads();
            // rows of the block: thread t owns [lo + t q2, lo + (t+1) q2)
            const int64_t lo = (int64_t)blk * R;
            const int64_t hi = lo + R < N ? lo + R : N;
            const int64_t q2 = (hi - lo + PICK_THREADS - 1) / PICK_THREADS;
            const int64_t r0 = lo + t * q2, r1 = r0 + q2 < hi ? r0 + q2 : hi;
            double lw = 0.0;
            for (int64_t i = r0; i < r1; ++i) lw = __dadd_rn(lw, w[i]);
            double Wb;
            const double ex2 = block_exclusive_scan(lw, buf, &Wb);
            double run2 = __dadd_rn(s_base, ex2);
            for (int64_t i = r0; i < r1; ++i) {
                const double wi = w[i];
                const double nxt = __dadd_rn(run2, wi);
                if (wi > 0.0) {
                    atomicMax(&s_last, (long long)i);
                    if (found && nxt > target) {
                        atomicMin(&s_pick, (long long)i);
                        break;
                    }
                }
                run2 = nxt;
            }
            __syncthreads();
            pick = s_pick != LLONG_MAX ? (int64_t)s_pick : (s_last >= 0 ? (int64_t)s_last : uniform_row(uc, N));
        }
    }
    if (t == 0) idx[c] = (int32_t)pick;
    for (int k = t; k < d; k += blockDim.x) C[(size_t)c * d + k] = X[(size_t)pick * d + k];
}

template <typename T>
cudaError_t seed_launches(const T* X, int64_t N, int d, int K, T* C, int32_t* idx, const double* u, double* w,
                          double* P, int NB, int64_t R, cudaStream_t s)
{
    k_pp_pick<T><<<1, PICK_THREADS, 0, s>>>(X, N, d, C, idx, u, 0, w, P, NB, R);
    for (int c = 1; c < K; ++c) {
        k_pp_weights<T><<<NB, PP_THREADS, 0, s>>>(X, N, d, C, c, R, w, P);
        k_pp_pick<T><<<1, PICK_THREADS, 0, s>>>(X, N, d, C, idx, u, c, w, P, NB, R);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace km

using namespace km;

extern "C" kmeans_status kmeans_seed_pp(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const double* u_host,
                                        void* C_out, int32_t* idx_out)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, false);
    if (s != KM_OK) return s;
    if (!u_host || !C_out) return fail(ctx, KM_EINVAL, "u_host and C_out must not be NULL");
    if (X->N > (int64_t)INT32_MAX) return fail(ctx, KM_EINVAL, "row indices are int32: N must be below 2^31");
    for (int k = 0; k < K; ++k)
        if (!(u_host[k] >= 0.0 && u_host[k] < 1.0)) return fail(ctx, KM_EINVAL, "every u must lie in [0, 1)");
    KM_CUDA(cudaSetDevice(ctx->device));
    const int64_t N = X->N;
    int64_t NB = (N + PICK_THREADS - 1) / PICK_THREADS;
    const int64_t cap = (int64_t)ctx->nsm * 8;
    if (NB > cap) NB = cap;
    if (NB < 1) NB = 1;
    const int64_t R = (N + NB - 1) / NB;
    NB = (N + R - 1) / R;                            // no empty block
    size_t o = 256;                                  // offset 0 holds the per-call counter
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) / 256 * 256; return r; };
    const size_t ow = take((size_t)N * 8), oP = take((size_t)NB * 8), ou = take((size_t)K * 8),
                 oi = take((size_t)K * 4);
    if ((s = ensure_arena(ctx, o)) != KM_OK) return s;
    char* base = arena_base(ctx);
    double* w = reinterpret_cast<double*>(base + ow);
    double* P = reinterpret_cast<double*>(base + oP);
    double* u = reinterpret_cast<double*>(base + ou);
    int32_t* idx = idx_out ? idx_out : reinterpret_cast<int32_t*>(base + oi);
    KM_CUDA(cudaMemcpyAsync(u, u_host, (size_t)K * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (X->prec == KM_F64)
        KM_CUDA(seed_launches(reinterpret_cast<const double*>(X->X), N, X->d, K, reinterpret_cast<double*>(C_out),
                              idx, u, w, P, (int)NB, R, ctx->stream));
    else
        KM_CUDA(seed_launches(reinterpret_cast<const float*>(X->X), N, X->d, K, reinterpret_cast<float*>(C_out), idx,
                              u, w, P, (int)NB, R, ctx->stream));
    return KM_OK;
}
