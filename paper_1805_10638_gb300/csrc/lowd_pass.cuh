// Templates of the low-d assignment pass (see lowd_pass.cu for what one pass computes).  Each
// instantiation unit (lowd_inst.cuh) includes this header for one precision and one of the
// standalone / batched kernels, so that the four sets compile in parallel.
#pragma once

#include "controller.cuh"
#include "km_internal.cuh"
#include "lowd_inst.cuh"

#include <type_traits>

namespace km {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int W = LOWD_THREADS / 32;

__device__ __forceinline__ float fmin3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Centroids per argmin chunk of the FP32 scan with few dimensions (8 or 16; both divide KPAD_ALIGN).
#ifndef KM_LOWD_CHUNK_SMALL
#define KM_LOWD_CHUNK_SMALL 8
#endif

__host__ __device__ constexpr int chunk_of(int D) { return D <= 8 ? KM_LOWD_CHUNK_SMALL : 8; }

template <int D>
struct Shape {
    static constexpr int DP = ((2 * (D + 1) + 3) / 4 * 4) / 2;   // packed floats per centroid
    static constexpr int R = (D <= 8) ? 4 : 2;             // samples per thread in the scan
    static constexpr int CK = chunk_of(D);                 // centroids per argmin chunk
};

// Resident blocks per SM the compiler must allow (register budget): the FP32 scan with few
// dimensions is latency-bound at 2 blocks per SM (16 warps), so it is compiled for 3 (85 registers,
// no spills up to d = 3; at 4 blocks the 64-register cap spills the bounds and bins code).
#ifndef KM_LOWD_MINB_SMALL
#define KM_LOWD_MINB_SMALL 3
#endif
#ifndef KM_LOWD_MINB_LARGE
#define KM_LOWD_MINB_LARGE 2
#endif
template <typename T, int D>
struct MinBlocks {
    static constexpr int value =
        std::is_same<T, float>::value ? (D <= 8 ? KM_LOWD_MINB_SMALL : KM_LOWD_MINB_LARGE) : 1;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

struct Layout {
    size_t red, org, cpk, rec, c, stage, bS, bC, hdr, hs, hm, hq, gd, gperm, goff, total;
};

// Skewed copy of the packed centroids for the per-row recovery reads: chunk b (CK centroids of
// D+1 floats) starts at b * RS floats, RS = CK(D+1)+1 is odd, so lanes recovering different chunks
// read different banks (the unskewed layout puts every chunk's element (q,k) in the same bank).
__host__ __device__ constexpr int rec_stride_of(int D) { return chunk_of(D) * (D + 1) + 1; }
template <int D>
__host__ __device__ constexpr int rec_stride() { return rec_stride_of(D); }

// hq_cap > 0 (FP32 passes with Hamerly bounds): centroid drifts, half distances to the nearest other
// centroid, drift maxima and the queue of rows that need a full scan.
// bins: the per-cluster residual sums of the update.  Per warp in the element type (sums combined in
// a fixed order), or with fx, once per block as 64-bit fixed point (exact, order-independent adds).
__host__ __device__ inline Layout layout(bool f32, int D, int DP, int K, int Kpad, bool bins, int hq_cap = 0,
                                         bool fx = false, int hg = 0)
{
    const size_t esz = f32 ? 4 : 8;
    Layout L;
    size_t o = 0;
    L.red = o;   o += 64 * sizeof(double);
    L.org = o;   o += 64 * sizeof(float);
    if (f32) {
        L.cpk = o; o += al16((size_t)Kpad * DP * 4);
        L.rec = o; o += al16((size_t)(Kpad / chunk_of(D)) * rec_stride_of(D) * 4);
        L.c = o;   o += al16((size_t)K * D * 4);
    } else {
        L.cpk = 0;
        L.rec = 0;
        L.c = o;   o += al16((size_t)K * D * 8);
    }
    L.stage = o; o += al16((size_t)W * 32 * D * esz);
    if (bins && fx) {
        L.bS = o; o += al16((size_t)K * D * 8);
        L.bC = o; o += al16((size_t)K * 4);
    } else if (bins) {
        L.bS = o; o += al16((size_t)W * K * D * esz);
        L.bC = o; o += al16((size_t)W * K * 4);
    } else {
        L.bS = L.bC = 0;
    }
    if (f32 && hq_cap > 0) {
        L.hdr = o; o += al16((size_t)Kpad * 4);
        L.hs = o;  o += al16((size_t)Kpad * 4);
        L.hm = o;  o += 16 * 4;
        L.hq = o;  o += al16((size_t)hq_cap * 4);
    } else {
        L.hdr = L.hs = L.hm = L.hq = 0;
    }
    if (f32 && hq_cap > 0 && hg > 0) {   // group bounds: group drifts, centroids in group order, offsets
        L.gd = o;    o += al16((size_t)hg * 4);
        L.gperm = o; o += al16((size_t)K * 4);
        L.goff = o;  o += al16((size_t)(hg + 1) * 4);
    } else {
        L.gd = L.gperm = L.goff = 0;
    }
    L.total = o;
    return L;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Block-wide fixed-order sums (result valid in thread 0).
__device__ double block_sum_d(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}
__device__ long long block_sum_ll(long long v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long* r = reinterpret_cast<long long*>(red);
    v = warp_sum_ll(v);
    __syncthreads();
    if (lane == 0) r[warp] = v;
    __syncthreads();
    long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += r[w];
    __syncthreads();
    return s;
}

// Minimum of one chunk's scores (pairs of centroids), by 3-input min instructions.
__device__ __forceinline__ float chunk_min(const float2 (&s)[4])
{
    return fmin3f(fmin3f(s[0].x, s[0].y, s[1].x), fmin3f(s[1].y, s[2].x, s[2].y), fminf(s[3].x, s[3].y));
}
__device__ __forceinline__ float chunk_min(const float2 (&s)[8])
{
    const float a = fmin3f(s[0].x, s[0].y, s[1].x), b = fmin3f(s[1].y, s[2].x, s[2].y);
    const float c = fmin3f(s[3].x, s[3].y, s[4].x), d = fmin3f(s[4].y, s[5].x, s[5].y);
    const float e = fmin3f(s[6].x, s[6].y, s[7].x);
    return fminf(fmin3f(a, b, c), fmin3f(d, e, s[7].y));
}

// Scan all centroids for R samples: per chunk of CK centroids (CK/2 interleaved pairs), each
// fma.rn.f32x2 scores one sample against two centroids; xd holds each sample coordinate twice.
template <int D, int R>
__device__ __forceinline__ void scan_chunks(const float* __restrict__ s_cpk, int Kpad,
                                            const float2 (&xd)[R][D], float (&best)[R],
                                            float (&sec)[R], int (&bc)[R])
{
    constexpr int PP = 2 * Shape<D>::DP;        // floats per centroid pair
    constexpr int CK = Shape<D>::CK;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        best[r] = __int_as_float(0x7f800000);
        sec[r] = __int_as_float(0x7f800000);
        bc[r] = 0;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < Kpad; c0 += CK) {
        float2 s[R][CK / 2];
#pragma unroll
        for (int p = 0; p < CK / 2; ++p) {
            float cv[PP];
            const float4* p4 = reinterpret_cast<const float4*>(s_cpk + (size_t)((c0 >> 1) + p) * PP);
#pragma unroll
            for (int v = 0; v < PP / 4; ++v) {
                const float4 t = p4[v];
                cv[4 * v] = t.x;
                cv[4 * v + 1] = t.y;
                cv[4 * v + 2] = t.z;
                cv[4 * v + 3] = t.w;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 acc = make_float2(cv[2 * D], cv[2 * D + 1]);
#pragma unroll
                for (int k = 0; k < D; ++k) acc = __ffma2_rn(make_float2(cv[2 * k], cv[2 * k + 1]), xd[r][k], acc);
                s[r][p] = acc;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float m = chunk_min(s[r]);
            sec[r] = fminf(sec[r], fmaxf(best[r], m));
            const bool p = m < best[r];
            best[r] = p ? m : best[r];
            bc[r] = p ? c0 : bc[r];
        }
    }
}

// Re-score the best chunk with the same arithmetic; lowest index attaining `best` and the
// smallest other value in the chunk.
template <int D>
__device__ __forceinline__ int recover(const float* __restrict__ s_rec, const float (&x)[D], float best,
                                       int bc, float& second_in)
{
    constexpr int RS = rec_stride<D>();
    constexpr int CK = Shape<D>::CK;
    const float* base = s_rec + (size_t)(bc / CK) * RS;
    int jj = -1;
    float sv = __int_as_float(0x7f800000);
#pragma unroll
    for (int q = 0; q < CK; ++q) {
        const float* cp = base + q * (D + 1);
        float acc = cp[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc = fmaf(cp[k], x[k], acc);
        if (acc == best && jj < 0)
            jj = q;
        else
            sv = fminf(sv, acc);
    }
    second_in = sv;
    if (jj < 0) {                 // cannot happen with identical arithmetic; force a rescore
        second_in = -__int_as_float(0x7f800000);
        return bc;
    }
    return bc + jj;
}

// Warp-cooperative FP32 direct-form rescoring of the rows some lanes flagged: for each flagged
// row in turn, the 32 lanes split the K centroids (ascending j per lane, strict '<'), then a
// lexicographic (distance, index) butterfly gives the lowest index attaining the minimum.
template <int D>
__device__ __forceinline__ int warp_rescore(const float* __restrict__ s_c32, int K, const float* __restrict__ X,
                                            int64_t my_row, bool need, int idx, int lane, long long& resc)
{
    unsigned bal = __ballot_sync(FULL, need);
    while (bal) {
        const int l = __ffs(bal) - 1;
        bal &= bal - 1;
        const int64_t row = __shfl_sync(FULL, my_row, l);
        float xo[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xo[k] = X[row * D + k];
        float bd = __int_as_float(0x7f800000);
        int bj = K;
        for (int j = lane; j < K; j += 32) {
            const float* c = s_c32 + (size_t)j * D;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = xo[k] - c[k];
                acc = fmaf(t, t, acc);
            }
            if (acc < bd) {
                bd = acc;
                bj = j;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(FULL, bd, o);
            const int oj = __shfl_xor_sync(FULL, bj, o);
            if (ob < bd || (ob == bd && oj < bj)) {
                bd = ob;
                bj = oj;
            }
        }
        if (lane == l) {
            idx = bj;
            resc += 1;
        }
    }
    return idx;
}

// Per-pass inputs of the Hamerly bounds of one solve: computed by k_hprep before the INIT and
// TRIAL passes (on C^0, C^t; the half distances split over its blocks), and by the TRIAL pass's
// last block alone for the REVERT pass (on C_AU) when the safeguard fired.  All in FP32 with explicit margins so that they only loosen the
// bounds:
//   hdr[j] = ||c_j - c_j^last|| (1 + 1e-5) + eta      drift since the centroids of the last pass
//   hs[j]  = (min_{j' != j} ||c_j - c_j'|| / 2)(1 - 1e-5) - eta, at least 0
//   hm     = (largest drift, second largest, index of the largest, eta)
// with eta = 4e-7 max(||c||, ||c^last||), the allowance for the rounding of the FP32 centroids.
// Block `part` of `nparts`: every block computes eta, all drifts and their top two (O(K d), so no
// block waits for another); the half distances, O(K^2 d), are split: block `part` takes the
// centroids [part*K/nparts, (part+1)*K/nparts).  Block 0 writes hdr and hm.
template <int D>
__device__ void hprep_body(const PassArgs& a, int mode, float* s_r, int part = 0, int nparts = 1)
{                                                                     // s_r: 96 floats of block scratch
    const SolveState* st = a.st;
    if (st->done) return;
    int which = 0;
    if (mode == MODE_REVERT) {
        if (!st->revert) return;
        which = 1;
    }
    constexpr int d = D;
    const int K = a.K, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const float* cs = a.c32[which];
    const float* cl = a.hlast;
    const bool have_last = mode != MODE_INIT;
    const bool writer = part == 0;
    __syncthreads();      // s_r may be in use by the caller's previous step
    float cm = 0.f;
    for (int j = tid; j < K; j += blockDim.x) {
        float n1 = 0.f, n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            n1 = fmaf(cs[j * d + k], cs[j * d + k], n1);
            if (have_last) n2 = fmaf(cl[j * d + k], cl[j * d + k], n2);
        }
        cm = fmaxf(cm, fmaxf(n1, n2));
    }
    for (int off = 16; off > 0; off >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, off));
    if (lane == 0) s_r[warp] = cm;
    __syncthreads();
    if (warp == 0) {
        cm = lane < nw ? s_r[lane] : 0.f;
        for (int off = 16; off > 0; off >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, off));
        if (lane == 0) s_r[32] = cm;
    }
    __syncthreads();
    const float eta = 4e-7f * sqrtf(s_r[32]) + 1e-30f;
    __syncthreads();
    // drifts of all centroids and their top two (every block; block 0 writes them)
    float m1 = 0.f, m2 = 0.f;
    int i1 = -1;
    if (have_last) {
        for (int j = tid; j < K; j += blockDim.x) {
            float dd = 0.f;
            for (int k = 0; k < d; ++k) {
                const float t = cs[j * d + k] - cl[j * d + k];
                dd = fmaf(t, t, dd);
            }
            const float dr = sqrtf(dd) * (1.f + 1e-5f) + eta;
            if (writer) a.hdr[j] = dr;
            if (dr > m1) {
                m2 = m1;
                m1 = dr;
                i1 = j;
            } else if (dr > m2) {
                m2 = dr;
            }
        }
    } else if (writer) {
        for (int j = tid; j < K; j += blockDim.x) a.hdr[j] = 0.f;
    }
    if (a.hg > 0) {
        // group bounds: no half distances (their O(K^2 d) cost is what the groups avoid; 0 is a
        // valid, inactive value), and each group's largest drift, from the drifts written above
        if (!writer) return;
        for (int j = tid; j < K; j += blockDim.x) a.hs[j] = 0.f;
        __syncthreads();
        for (int gi = tid; gi < a.hg; gi += blockDim.x) {
            float mx = 0.f;
            if (have_last)
                for (int p = a.hgoff[gi]; p < a.hgoff[gi + 1]; ++p) mx = fmaxf(mx, a.hdr[a.hperm[p]]);
            a.hgd[gi] = mx;
        }
    } else {
    // half distances of this block's centroids: tpj consecutive lanes share a centroid j and split
    // the j2 range.  The outer trip count is the same for every thread (lanes past the range compute
    // nothing) because the lanes of a centroid combine their minima with warp shuffles.
    const int jlo = (int)((long long)K * part / nparts), jhi = (int)((long long)K * (part + 1) / nparts);
    const int nj = jhi - jlo;
    int tpj = 1;
    while (tpj < 32 && 2 * tpj * nj <= (int)blockDim.x) tpj <<= 1;
    const int sub = tid % tpj, per = blockDim.x / tpj;
    for (int jb = 0; jb < nj; jb += per) {
        const int j = jlo + jb + tid / tpj;
        const bool valid = j < jhi;
        const int jc = valid ? j : jlo;
        float cj[D];
#pragma unroll
        for (int k = 0; k < D; ++k) cj[k] = cs[jc * d + k];
        float mn = __int_as_float(0x7f800000);
#pragma unroll 4
        for (int j2 = sub; j2 < K; j2 += tpj) {
            float dd = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = cj[k] - __ldg(cs + j2 * d + k);
                dd = fmaf(t, t, dd);
            }
            mn = j2 == jc ? mn : fminf(mn, dd);
        }
        for (int off = 1; off < tpj; off <<= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        if (valid && sub == 0) a.hs[j] = fmaxf(0.f, 0.5f * sqrtf(mn) * (1.f - 1e-5f) - eta);
    }
    }
    if (!writer) return;
    for (int off = 16; off > 0; off >>= 1) {
        const float om1 = __shfl_xor_sync(0xffffffffu, m1, off), om2 = __shfl_xor_sync(0xffffffffu, m2, off);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, off);
        if (om1 > m1) {
            m2 = fmaxf(m1, om2);
            m1 = om1;
            i1 = oi1;
        } else {
            m2 = fmaxf(m2, om1);
        }
    }
    if (lane == 0) {
        s_r[3 * warp] = m1;
        s_r[3 * warp + 1] = m2;
        s_r[3 * warp + 2] = __int_as_float(i1);
    }
    __syncthreads();
    if (warp == 0) {                 // the warps' top two, merged the same way
        m1 = lane < nw ? s_r[3 * lane] : 0.f;
        m2 = lane < nw ? s_r[3 * lane + 1] : 0.f;
        i1 = lane < nw ? __float_as_int(s_r[3 * lane + 2]) : -1;
        for (int off = 16; off > 0; off >>= 1) {
            const float om1 = __shfl_xor_sync(0xffffffffu, m1, off), om2 = __shfl_xor_sync(0xffffffffu, m2, off);
            const int oi1 = __shfl_xor_sync(0xffffffffu, i1, off);
            if (om1 > m1) {
                m2 = fmaxf(m1, om2);
                m1 = om1;
                i1 = oi1;
            } else {
                m2 = fmaxf(m2, om1);
            }
        }
        if (lane == 0) {
            a.hm[0] = m1;
            a.hm[1] = m2;
            a.hm[2] = __int_as_float(i1);
            a.hm[3] = eta;
        }
    }
}


#define KM_HPREP_CASE(DD) \
    case DD:              \
        hprep_body<DD>(a, mode, s_r, part, nparts); \
        break;

// k_hprep / k_hprep_batch: the block's instance has its dimension at run time.
__device__ inline void hprep_dispatch(const PassArgs& a, int mode, float* s_r, int part = 0, int nparts = 1)
{
    switch (a.d) {
        KM_FOR_EACH_D(KM_HPREP_CASE)
        default:
            break;
    }
}

// Group bounds after a full scan settled row x on centroid idx: per group the FP32 direct-form
// distance to its nearest centroid other than idx, lowered by the margins that raise the upper bound
// (relative 1e-5 and the absolute eta), written to lr[0..hg).  Kept out of line: only scanned rows
// take it, and the pass's main loops keep their registers.
template <int D>
__device__ __noinline__ void group_lower_bounds(const float* xr, int idx, const float* c, const int* perm,
                                                const int* goff, int hg, float eta, float* lr)
{
    float x[D];
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = xr[k];
    for (int gi = 0; gi < hg; ++gi) {
        float mn = __int_as_float(0x7f800000);
        for (int p = goff[gi]; p < goff[gi + 1]; ++p) {
            const int j = perm[p];
            const float* cj = c + (size_t)j * D;
            float d2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = x[k] - cj[k];
                d2 = fmaf(t, t, d2);
            }
            mn = j == idx ? mn : fminf(mn, d2);
        }
        lr[gi] = fmaxf(0.f, sqrtf(mn) * (1.f - 1e-5f) - eta);
    }
}

// Phase A of a pass with group bounds, for this thread's rows: the assigned centroid a is kept if its
// upper bound u (plus a's drift since the last pass) is below the smallest group lower bound, each
// lowered by its group's largest drift, by a relative margin of 1e-5; failing that, the test is
// retried with u recomputed as the exact distance to a.  Kept rows get the new u and the lowered
// group bounds; the others are queued for a full scan.  Returns the number queued.
// Rows are taken from *cursor on; when the queue (capacity cap) is full the thread stops at the row it
// could not queue and the caller drains the queue before the next round.
template <int D>
__device__ __noinline__ long long group_classify(const PassArgs& a, const float* X, int64_t g, int64_t TT, int64_t n_g,
                                                 int64_t* cursor, unsigned cap, bool force, const int32_t* rho_last,
                                                 int32_t* rho_out, const float* s_hdr, const float* s_gd,
                                                 const float* c, float eta, int hg, uint32_t* s_hq,
                                                 unsigned int* s_hqn, bool chk, int* bad, float* xabs)
{
    long long nq = 0;
    for (int64_t q = *cursor; q < n_g; ++q) {
        const int64_t row = g + q * TT;
        float xv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xv[k] = X[row * D + k];
        if (chk) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                *bad |= !isfinite(xv[k]);
                *xabs = fmaxf(*xabs, fabsf(xv[k]));
            }
        }
        bool scan = force;
        if (!force) {
            const int a_ = rho_last[row];
            float u = (a.hub[row] + s_hdr[a_]) * (1.f + 2e-7f);
            float* lr = a.hlbg + (size_t)row * hg;
            float m = __int_as_float(0x7f800000);
            for (int gi = 0; gi < hg; ++gi) m = fminf(m, fmaxf(0.f, (lr[gi] - s_gd[gi]) * (1.f - 2e-7f)));
            if (!(u * (1.f + 1e-5f) < m)) {
                const float* ca = c + (size_t)a_ * D;
                float dd = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float t = xv[k] - ca[k];
                    dd = fmaf(t, t, dd);
                }
                u = sqrtf(dd) * (1.f + 1e-5f) + eta;
                scan = !(u * (1.f + 1e-5f) < m);
            }
            if (!scan) {
                rho_out[row] = a_;
                a.hub[row] = u;
                for (int gi = 0; gi < hg; ++gi) lr[gi] = fmaxf(0.f, (lr[gi] - s_gd[gi]) * (1.f - 2e-7f));
            }
        }
        if (scan) {
            const unsigned pos = atomicAdd(s_hqn, 1u);
            if (pos >= cap) {               // full: this row again in the next round
                *cursor = q;
                return nq;
            }
            s_hq[pos] = (uint32_t)row;
            nq += 1;
        }
    }
    *cursor = n_g;
    return nq;
}

// The work of block `bid` of a pass launched with `nblk` blocks.  The standalone kernel calls it
// with (blockIdx.x, gridDim.x); the batched kernel with a work item's (block, blocks of that
// instance), so that every instance gets exactly the arithmetic of its own launch.
// RV: rows per thread of the FP32 scan (0: Shape<D>::R).  Each row's scan and the order in which
// rows are finished do not depend on it, so every RV gives bitwise the same results.
// AO: a pass without update bins and without bounds (the standalone assignment and energy calls):
// that code is compiled out, so the kernel fits a tighter register budget.
template <typename T, int D, int RV = 0, bool AO = false>
__device__ __forceinline__ void pass_body(const PassArgs& a, const int bid, const int nblk, unsigned char* smem)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int DP = Shape<D>::DP;
    constexpr int R = F32 ? (RV > 0 ? RV : Shape<D>::R) : 1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    SolveState* st = a.st;
    int which = 0;
    int32_t* rho_out = a.rho[0];
    const int32_t* rho_prev = a.rho_prev;
    const int32_t* rho_in = a.rho_in;
    if (a.mode == MODE_EPI) {
        // energy of (P^t, G^t) when the loop stopped at max_iter
        if (st->converged || st->status != KM_OK) return;
        which = 1;
        rho_in = a.rho[st->cur];
    } else if (a.mode != MODE_STANDALONE) {
        if (st->done) return;
        if (a.mode == MODE_REVERT) {
            if (!st->revert) return;
            which = 1;
        }
        const int cur = st->cur;
        rho_out = a.rho[cur];
        rho_prev = (a.mode == MODE_INIT) ? nullptr : a.rho[cur ^ 1];
    }
    const int flags = a.flags;
    const bool do_assign = flags & F_ASSIGN;
    const bool do_bins = !AO && (flags & F_BINS);
    const int K = a.K;
    // Hamerly bounds: FP32 solver passes that assign (INIT computes the bounds, TRIAL and REVERT use them)
    const bool ham = !AO && F32 && a.ham && do_assign &&
                     (a.mode == MODE_INIT || a.mode == MODE_TRIAL || a.mode == MODE_REVERT);
    // the solver's TRIAL / REVERT update sums in 64-bit fixed point (see layout)
    const bool fx = F32 && D <= FX_MAX_D && do_bins && a.acc != nullptr &&
                    (a.mode == MODE_TRIAL || a.mode == MODE_REVERT);
    const Layout L = layout(F32, D, DP, K, a.Kpad, do_bins, a.ham ? a.hq_cap : 0, fx, a.ham ? a.hg : 0);
    double* s_red = reinterpret_cast<double*>(smem + L.red);
    T* s_stage = reinterpret_cast<T*>(smem + L.stage);
    T* s_bS = reinterpret_cast<T*>(smem + L.bS);
    int* s_bC = reinterpret_cast<int*>(smem + L.bC);
    const float* s_cpk = reinterpret_cast<const float*>(smem + L.cpk);
    const T* s_c = reinterpret_cast<const T*>(smem + L.c);

    // ---- stage centroids and clear bins
    const float* s_rec = reinterpret_cast<const float*>(smem + L.rec);
    float* s_org = reinterpret_cast<float*>(smem + L.org);
    if constexpr (F32) {
        float* dst = reinterpret_cast<float*>(smem + L.cpk);
        float* dc = reinterpret_cast<float*>(smem + L.c);
        if (flags & F_PACK) {
            // standalone call: o = mean of the given centroids (a shift that only keeps the FP32
            // scores small; FP32 sums in a fixed order: per thread, butterfly, warps in order), then pack
            const float* Cr = a.rawC;
            float ov[D];
#pragma unroll
            for (int k = 0; k < D; ++k) ov[k] = 0.f;
            for (int j = tid; j < K; j += blockDim.x)
#pragma unroll
                for (int k = 0; k < D; ++k) ov[k] += Cr[(size_t)j * D + k];
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) ov[k] += __shfl_xor_sync(FULL, ov[k], off);
            float* fr = reinterpret_cast<float*>(s_red);        // [W][D] <= 128 floats
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < D; ++k) fr[warp * D + k] = ov[k];
            __syncthreads();
            if (tid < D) {
                float v = 0.f;
                for (int w = 0; w < W; ++w) v += fr[w * D + tid];
                s_org[tid] = v / (float)K;
            }
            __syncthreads();
            for (int j = tid; j < a.Kpad; j += blockDim.x) {
#pragma unroll
                for (int k = 0; k < DP; ++k) dst[pk_index(j, k, DP)] = 0.f;
                if (j < K) {
                    double nrm = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float c = Cr[(size_t)j * D + k];
                        dc[(size_t)j * D + k] = c;
                        const float cc = c - s_org[k];           // rounded once, as in FP64 then FP32
                        dst[pk_index(j, k, DP)] = -2.f * cc;
                        nrm += (double)cc * (double)cc;
                    }
                    dst[pk_index(j, D, DP)] = (float)nrm;
                } else {
                    dst[pk_index(j, D, DP)] = __int_as_float(0x7f800000);
                }
            }
        } else {
            const float4* src = reinterpret_cast<const float4*>(a.cpk[which]);
            float4* dst4 = reinterpret_cast<float4*>(dst);
            for (int i = tid; i < a.Kpad * DP / 4; i += blockDim.x) dst4[i] = src[i];
            if (a.mode == MODE_EPI) {          // G^t was not packed: round it here
                const double* g64 = a.c64[1];
                for (int i = tid; i < K * D; i += blockDim.x) dc[i] = (float)g64[i];
            } else {
                const float* c32 = a.c32[which];
                for (int i = tid; i < K * D; i += blockDim.x) dc[i] = c32[i];
            }
            if (tid < D) s_org[tid] = a.origin[tid];
        }
    } else {
        const double* c64 = a.c64[which];
        double* dc = reinterpret_cast<double*>(smem + L.c);
        for (int i = tid; i < K * D; i += blockDim.x) dc[i] = c64[i];
    }
    if (do_bins && fx) {
        unsigned long long* fb = reinterpret_cast<unsigned long long*>(smem + L.bS);
        for (int i = tid; i < K * D; i += blockDim.x) fb[i] = 0ull;
        for (int i = tid; i < K; i += blockDim.x) s_bC[i] = 0;
    } else if (do_bins) {
        for (int i = tid; i < W * K * D; i += blockDim.x) s_bS[i] = T(0);
        for (int i = tid; i < W * K; i += blockDim.x) s_bC[i] = 0;
    }
    __syncthreads();

    // ---- skewed recovery copy and the rounding-error bound's max|c'| (FP32 path)
    float cmax = 0.f;
    float o[D];
    if constexpr (F32) {
        constexpr int RS = rec_stride<D>();
        float* sr = reinterpret_cast<float*>(smem + L.rec);
        for (int i = tid; i < a.Kpad * (D + 1); i += blockDim.x) {
            const int j = i / (D + 1), k = i % (D + 1);
            sr[(size_t)(j / Shape<D>::CK) * RS + (j % Shape<D>::CK) * (D + 1) + k] = s_cpk[pk_index(j, k, DP)];
        }
        float mx = 0.f;
        for (int j = tid; j < K; j += blockDim.x) mx = fmaxf(mx, s_cpk[pk_index(j, D, DP)]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
        float* fr = reinterpret_cast<float*>(s_red);
        if (lane == 0) fr[warp] = mx;
        __syncthreads();
        mx = 0.f;
        for (int w = 0; w < W; ++w) mx = fmaxf(mx, fr[w]);
        cmax = sqrtf(mx);
#pragma unroll
        for (int k = 0; k < D; ++k) o[k] = s_org[k];
        __syncthreads();
    }

    // ---- Hamerly: the per-pass inputs k_hprep wrote (drifts, half distances, drift maxima, eta)
    float h_eta = 0.f, h_dm1 = 0.f, h_dm2 = 0.f;
    int h_am = -1;
    float* s_hdr = reinterpret_cast<float*>(smem + L.hdr);
    float* s_hs = reinterpret_cast<float*>(smem + L.hs);
    float* s_hm = reinterpret_cast<float*>(smem + L.hm);
    unsigned int* s_hqn = reinterpret_cast<unsigned int*>(s_hm + 8);
    uint32_t* s_hq = reinterpret_cast<uint32_t*>(smem + L.hq);
    const int HG = ham ? a.hg : 0;               // groups of the group bounds (0: Hamerly)
    float* s_gd = reinterpret_cast<float*>(smem + L.gd);
    int* s_gperm = reinterpret_cast<int*>(smem + L.gperm);
    int* s_goff = reinterpret_cast<int*>(smem + L.goff);
    if constexpr (F32) {
        if (ham) {
            for (int jj = tid; jj < K; jj += blockDim.x) {
                s_hdr[jj] = a.hdr[jj];
                s_hs[jj] = a.hs[jj];
            }
            if (HG > 0) {
                for (int jj = tid; jj < K; jj += blockDim.x) s_gperm[jj] = a.hperm[jj];
                for (int gi = tid; gi <= HG; gi += blockDim.x) s_goff[gi] = a.hgoff[gi];
                for (int gi = tid; gi < HG; gi += blockDim.x) s_gd[gi] = a.hgd[gi];
            }
            if (tid == 0) *s_hqn = 0u;
            __syncthreads();
            h_dm1 = a.hm[0];
            h_dm2 = a.hm[1];
            h_am = __float_as_int(a.hm[2]);
            h_eta = a.hm[3];
        }
    }

    // fixed-point scale 2^fx_s: every residual |r_k| <= max|x| + max|c|, so N of them stay below 2^61
    float fx_f = 0.f;
    int fx_s = 0;
    if constexpr (F32) {
        if (fx) {
            float cm = 0.f;
            for (int i = tid; i < K * D; i += blockDim.x) cm = fmaxf(cm, fabsf(reinterpret_cast<const float*>(s_c)[i]));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cm = fmaxf(cm, __shfl_xor_sync(FULL, cm, off));
            float* fr = reinterpret_cast<float*>(s_red);
            __syncthreads();
            if (lane == 0) fr[warp] = cm;
            __syncthreads();
            cm = 0.f;
            for (int w = 0; w < W; ++w) cm = fmaxf(cm, fr[w]);
            __syncthreads();
            const double rb = ((double)st->xmax + (double)cm) * (double)a.N;
            fx_s = rb > 0.0 ? 60 - ilogb(rb) : 0;
            fx_s = fx_s > 100 ? 100 : (fx_s < -100 ? -100 : fx_s);
            fx_f = ldexpf(1.f, fx_s);
        }
    }

    const T* X = reinterpret_cast<const T*>(a.X);
    const int64_t N = a.N;
    const int64_t TT = (int64_t)nblk * blockDim.x;
    const int64_t g = (int64_t)bid * blockDim.x + tid;
    const int64_t n_g = g < N ? (N - 1 - g) / TT + 1 : 0;
    const int64_t n_min = __shfl_sync(FULL, n_g, 31);
    const int64_t n_max = __shfl_sync(FULL, n_g, 0);

    T eacc = T(0);
    long long nch = 0, resc = 0, nscan = 0;
    int bad = 0;

    // Everything after the label is known, for one sample (warp-uniform call).
    // xr: the sample (global memory or preloaded registers); prev: its previous label, or -2 to
    // read it here.
    auto finish_x = [&](int64_t row, bool valid, int idx, const T* xr, int prev) {
        idx = idx < K ? idx : K - 1;           // only reachable with non-finite data
        T res[D];
        T e = T(0);
        if (valid) {
            const T* c = s_c + (size_t)idx * D;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if constexpr (F32) {
                    res[k] = xr[k] - c[k];
                    e = fmaf(res[k], res[k], e);
                } else {
                    res[k] = __dsub_rn(xr[k], c[k]);
                    e = __dadd_rn(e, __dmul_rn(res[k], res[k]));
                }
            }
            if (do_assign) rho_out[row] = idx;
            if ((flags & F_CHANGED) && rho_prev) nch += ((prev == -2 ? rho_prev[row] : prev) != idx);
            if (flags & F_DMIN) reinterpret_cast<T*>(a.dmin)[row] = e;
            eacc += e;
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) res[k] = T(0);
        }
        if (do_bins && fx) {
            if (valid) {
                unsigned long long* fb = reinterpret_cast<unsigned long long*>(s_bS) + (size_t)idx * D;
#pragma unroll
                for (int k = 0; k < D; ++k)
                    atomicAdd(fb + k, (unsigned long long)__float2ll_rn((float)res[k] * fx_f));
                atomicAdd(s_bC + idx, 1);
            }
        } else if (do_bins) {
            const int lab = valid ? idx : -1;
            const unsigned mm = __match_any_sync(FULL, lab);
            T* stg = s_stage + (size_t)warp * 32 * D;
#pragma unroll
            for (int k = 0; k < D; ++k) stg[lane * D + k] = res[k];
            __syncwarp();
            if (valid && lane == __ffs(mm) - 1) {
                T acc[D];
#pragma unroll
                for (int k = 0; k < D; ++k) acc[k] = T(0);
                unsigned m2 = mm;
                while (m2) {
                    const int l = __ffs(m2) - 1;
                    m2 &= m2 - 1;
#pragma unroll
                    for (int k = 0; k < D; ++k) acc[k] += stg[l * D + k];
                }
                T* bin = s_bS + ((size_t)warp * K + lab) * D;
#pragma unroll
                for (int k = 0; k < D; ++k) bin[k] += acc[k];
                s_bC[warp * K + lab] += __popc(mm);
            }
            __syncwarp();
        }
    };

    auto finish = [&](int64_t row, bool valid, int idx) { finish_x(row, valid, idx, X + row * D, -2); };

    float xabs = 0.f;   // INIT pass (FP32 solver): max |x_ik| seen by this thread
    auto check = [&](const T* xr) {
        if (flags & F_CHECK) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                bad |= !isfinite(xr[k]);
                if constexpr (F32) xabs = fmaxf(xabs, fabsf((float)xr[k]));
            }
        }
    };

    int64_t kk = 0;
    if (do_assign) {
        if constexpr (F32) {
            const float cA = a.bound_coef, cB = a.bound_coef2;
            if (ham) {
                // Bounds of a row the full scan assigned: u from the exact FP32 distance to the chosen
                // centroid, l from the second-best score minus its error bound (0 after a near-tie
                // rescore, which is the conservative choice).
                auto ham_store = [&](int64_t row, int idx, float second, float xn, float bnd, bool rescored) {
                    const float* xr = X + row * D;
                    const float* c = reinterpret_cast<const float*>(s_c) + (size_t)idx * D;
                    float dd = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float t = xr[k] - c[k];
                        dd = fmaf(t, t, dd);
                    }
                    const float u = sqrtf(dd) * (1.f + 1e-5f) + h_eta;
                    float l = 0.f;
                    if (!rescored)
                        l = sqrtf(fmaxf(0.f, second - bnd + xn * (1.f - 2e-6f))) * (1.f - 1e-5f) - h_eta;
                    rho_out[row] = idx;
                    a.hub[row] = u;
                    a.hlb[row] = fmaxf(l, 0.f);
                    if (HG > 0)
                        group_lower_bounds<D>(xr, idx, reinterpret_cast<const float*>(s_c), s_gperm, s_goff, HG, h_eta,
                                              a.hlbg + (size_t)row * HG);
                };
                // phase A: rows whose bounds show the assigned centroid is still the unique nearest by
                // a relative margin of 1e-5 (far beyond the FP32 rounding of either score form, so a
                // full scan would return the same label) keep it; the others are queued
                const bool force = a.mode == MODE_INIT;
                const int32_t* rho_last = a.mode == MODE_TRIAL ? rho_prev : rho_out;
                constexpr int HB = 4;             // rows per thread whose loads are issued together
                // phases A and B run in rounds, so that a queue of hq_cap rows serves any number of
                // scans (the INIT pass scans every row).  Hamerly: a round classifies at most
                // hq_cap / blockDim.x rows per thread, so the queue cannot overflow; group bounds: a
                // thread whose row finds the queue full stops there and resumes after it is drained
                int64_t gcur = 0;
                const int64_t rpr = (int64_t)(a.hq_cap / (int)blockDim.x);
                for (int rnd = 0;; ++rnd) {
                if (HG > 0)
                    nscan += group_classify<D>(a, X, g, TT, n_g, &gcur, (unsigned)a.hq_cap, force, rho_last, rho_out,
                                               s_hdr, s_gd, reinterpret_cast<const float*>(s_c), h_eta, HG, s_hq,
                                               s_hqn, (flags & F_CHECK) != 0, &bad, &xabs);
                const int64_t qend = min(n_g, gcur + rpr);
                for (int64_t q0 = gcur; HG == 0 && q0 < qend; q0 += HB) {
                    int al[HB];
                    float ub[HB], lb[HB], xv[HB][D];
#pragma unroll
                    for (int r = 0; r < HB; ++r) {
                        const bool v = q0 + r < qend;
                        const int64_t row = g + (v ? q0 + r : q0) * TT;
                        al[r] = force ? 0 : rho_last[row];
                        ub[r] = force ? 0.f : a.hub[row];
                        lb[r] = force ? 0.f : a.hlb[row];
#pragma unroll
                        for (int k = 0; k < D; ++k) xv[r][k] = X[row * D + k];
                    }
#pragma unroll
                    for (int r = 0; r < HB; ++r) {
                        if (q0 + r >= qend) break;
                        const int64_t row = g + (q0 + r) * TT;
                        check(xv[r]);
                        bool scan = force;
                        if (!force) {
                            const int a_ = al[r];
                            float u = (ub[r] + s_hdr[a_]) * (1.f + 2e-7f);
                            const float l = fmaxf(0.f, (lb[r] - (a_ == h_am ? h_dm2 : h_dm1)) * (1.f - 2e-7f));
                            const float m = fmaxf(l, s_hs[a_]);
                            if (!(u * (1.f + 1e-5f) < m)) {
                                const float* c = reinterpret_cast<const float*>(s_c) + (size_t)a_ * D;
                                float dd = 0.f;
#pragma unroll
                                for (int k = 0; k < D; ++k) {
                                    const float t = xv[r][k] - c[k];
                                    dd = fmaf(t, t, dd);
                                }
                                u = sqrtf(dd) * (1.f + 1e-5f) + h_eta;
                                scan = !(u * (1.f + 1e-5f) < m);
                            }
                            if (!scan) {
                                rho_out[row] = a_;
                                a.hub[row] = u;
                                a.hlb[row] = l;
                            }
                        }
                        if (scan) {
                            s_hq[atomicAdd(s_hqn, 1u)] = (uint32_t)row;
                            nscan += 1;
                        }
                    }
                }
                if (HG == 0) gcur = qend;
                __syncthreads();
                // phase B: full scans of the queued rows, R per thread while whole rounds remain
                const int nq = (int)min(*s_hqn, (unsigned)a.hq_cap);
                const int round = (int)blockDim.x * R;
                int qb = 0;
                for (; qb + round <= nq; qb += round) {
                    int64_t rows[R];
                    float x[R][D];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        rows[r] = s_hq[qb + r * (int)blockDim.x + tid];
                        const float* xr = X + rows[r] * D;
#pragma unroll
                        for (int k = 0; k < D; ++k) x[r][k] = xr[k] - o[k];
                    }
                    float2 xd[R][D];
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int k = 0; k < D; ++k) xd[r][k] = make_float2(x[r][k], x[r][k]);
                    float best[R], sec[R];
                    int bc[R];
                    scan_chunks<D, R>(s_cpk, a.Kpad, xd, best, sec, bc);
                    int idxr[R];
                    bool need[R];
                    float sc2[R], xnr[R], bndr[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float xn = 0.f;
#pragma unroll
                        for (int k = 0; k < D; ++k) xn = fmaf(x[r][k], x[r][k], xn);
                        float sin_;
                        idxr[r] = recover<D>(s_rec, x[r], best[r], bc[r], sin_);
                        sc2[r] = fminf(sec[r], sin_);
                        xnr[r] = xn;
                        bndr[r] = cA * cmax * cmax + cB * sqrtf(xn) * cmax;
                        need[r] = sc2[r] - best[r] <= 2.f * bndr[r];
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        idxr[r] = warp_rescore<D>(reinterpret_cast<const float*>(s_c), K, X, rows[r], need[r], idxr[r],
                                                  lane, resc);
#pragma unroll
                    for (int r = 0; r < R; ++r) ham_store(rows[r], idxr[r], sc2[r], xnr[r], bndr[r], need[r]);
                }
                for (int e = qb + tid; e < qb + ((nq - qb + (int)blockDim.x - 1) / (int)blockDim.x) * (int)blockDim.x;
                     e += blockDim.x) {
                    const bool valid = e < nq;
                    const int64_t row = valid ? (int64_t)s_hq[e] : 0;
                    float x[1][D];
                    const float* xr = X + row * D;
#pragma unroll
                    for (int k = 0; k < D; ++k) x[0][k] = xr[k] - o[k];
                    float2 xd[1][D];
#pragma unroll
                    for (int k = 0; k < D; ++k) xd[0][k] = make_float2(x[0][k], x[0][k]);
                    float best[1], sec[1];
                    int bc[1];
                    scan_chunks<D, 1>(s_cpk, a.Kpad, xd, best, sec, bc);
                    float xn = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) xn = fmaf(x[0][k], x[0][k], xn);
                    float sin_;
                    int idx = recover<D>(s_rec, x[0], best[0], bc[0], sin_);
                    const float second = fminf(sec[0], sin_);
                    const float bnd = cA * cmax * cmax + cB * sqrtf(xn) * cmax;
                    const bool need = valid && second - best[0] <= 2.f * bnd;
                    idx = warp_rescore<D>(reinterpret_cast<const float*>(s_c), K, X, row, need, idx, lane, resc);
                    if (valid) ham_store(row, idx, second, xn, bnd, need);
                }
                __syncthreads();
                if (!__syncthreads_or(gcur < n_g)) break;
                if (tid == 0) *s_hqn = 0u;
                __syncthreads();
                }
                // phase C: the rest of the pass in the same per-thread row order as without bounds,
                // so the update's sums come out bitwise the same
                for (int64_t q0 = 0; q0 < n_max; q0 += HB) {
                    int lab[HB], prv[HB];
                    float xv[HB][D];
#pragma unroll
                    for (int r = 0; r < HB; ++r) {
                        const bool v = q0 + r < n_g;
                        const int64_t row = v ? g + (q0 + r) * TT : 0;
                        lab[r] = v ? rho_out[row] : 0;
                        prv[r] = (v && (flags & F_CHANGED) && rho_prev) ? rho_prev[row] : -1;
#pragma unroll
                        for (int k = 0; k < D; ++k) xv[r][k] = X[row * D + k];
                    }
#pragma unroll
                    for (int r = 0; r < HB; ++r) {
                        if (q0 + r >= n_max) break;
                        const bool v = q0 + r < n_g;
                        finish_x(v ? g + (q0 + r) * TT : 0, v, lab[r], xv[r], prv[r]);
                    }
                }
                kk = n_max;
            }
            const int64_t main_iters = ham ? 0 : n_min / R;
            if (!ham) nscan = n_g;
            for (int64_t it = 0; it < main_iters; ++it, kk += R) {
                float x[R][D];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float* xr = X + (g + (kk + r) * TT) * D;
                    check(xr);
#pragma unroll
                    for (int k = 0; k < D; ++k) x[r][k] = xr[k] - o[k];
                }
                float2 xd[R][D];
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int k = 0; k < D; ++k) xd[r][k] = make_float2(x[r][k], x[r][k]);
                float best[R], sec[R];
                int bc[R];
                scan_chunks<D, R>(s_cpk, a.Kpad, xd, best, sec, bc);
                int idxr[R];
                bool need[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float xn = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) xn = fmaf(x[r][k], x[r][k], xn);
                    float sin_;
                    idxr[r] = recover<D>(s_rec, x[r], best[r], bc[r], sin_);
                    const float second = fminf(sec[r], sin_);
                    const float bnd = cA * cmax * cmax + cB * sqrtf(xn) * cmax;
                    need[r] = second - best[r] <= 2.f * bnd;
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
                    idxr[r] = warp_rescore<D>(reinterpret_cast<const float*>(s_c), K, X, g + (kk + r) * TT, need[r],
                                              idxr[r], lane, resc);
#pragma unroll
                for (int r = 0; r < R; ++r) finish(g + (kk + r) * TT, true, idxr[r]);
            }
            for (; kk < n_max; ++kk) {
                const bool valid = kk < n_g;
                const int64_t row = valid ? g + kk * TT : 0;
                float x[1][D];
                const float* xr = X + row * D;
                if (valid) check(xr);
#pragma unroll
                for (int k = 0; k < D; ++k) x[0][k] = xr[k] - o[k];
                float2 xd[1][D];
#pragma unroll
                for (int k = 0; k < D; ++k) xd[0][k] = make_float2(x[0][k], x[0][k]);
                float best[1], sec[1];
                int bc[1];
                scan_chunks<D, 1>(s_cpk, a.Kpad, xd, best, sec, bc);
                float xn = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) xn = fmaf(x[0][k], x[0][k], xn);
                float sin_;
                int idx = recover<D>(s_rec, x[0], best[0], bc[0], sin_);
                const float second = fminf(sec[0], sin_);
                const float bnd = cA * cmax * cmax + cB * sqrtf(xn) * cmax;
                const bool need = valid && second - best[0] <= 2.f * bnd;
                idx = warp_rescore<D>(reinterpret_cast<const float*>(s_c), K, X, row, need, idx, lane, resc);
                finish(row, valid, idx);
            }
        } else {
            for (; kk < n_max; ++kk) {
                const bool valid = kk < n_g;
                const int64_t row = valid ? g + kk * TT : 0;
                const double* xr = X + row * D;
                if (valid) check(xr);
                double x[D];
#pragma unroll
                for (int k = 0; k < D; ++k) x[k] = xr[k];
                double bd = __longlong_as_double(0x7ff0000000000000LL);
                int bj = 0;
                for (int j = 0; j < K; ++j) {
                    const double* c = s_c + (size_t)j * D;
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const double t = __dsub_rn(x[k], c[k]);
                        s = __dadd_rn(s, __dmul_rn(t, t));
                    }
                    if (s < bd) {
                        bd = s;
                        bj = j;
                    }
                }
                finish(row, valid, bj);
            }
        }
    } else {
        // labels given: energy / update from rho_in
        for (; kk < n_max; ++kk) {
            const bool valid = kk < n_g;
            const int64_t row = valid ? g + kk * TT : 0;
            int idx = valid ? rho_in[row] : 0;
            idx = (idx >= 0 && idx < K) ? idx : 0;
            finish(row, valid, idx);
        }
    }

    // ---- block partials
    const double eb = block_sum_d((double)eacc, s_red);
    const long long nb_ch = block_sum_ll(nch, s_red);
    const long long nb_rs = block_sum_ll(resc, s_red);
    if constexpr (!F32) nscan = do_assign ? n_g : 0;
    const long long nb_sc = block_sum_ll(nscan, s_red);
    const long long nb_bad = block_sum_ll(bad, s_red);
    if (tid == 0) {
        a.pE[bid] = eb;
        a.pNch[bid] = nb_ch;
        a.pResc[bid] = nb_rs;
        if (a.pScan) a.pScan[bid] = nb_sc;
        a.pBad[bid] = (int)(nb_bad != 0);
    }
    if constexpr (F32) {
        if ((flags & F_CHECK) && a.mode == MODE_INIT) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) xabs = fmaxf(xabs, __shfl_xor_sync(FULL, xabs, off));
            if (lane == 0 && isfinite(xabs)) atomicMax(reinterpret_cast<int*>(&st->xmax), __float_as_int(xabs));
        }
    }
    if (do_bins && fx) {
        // integer adds into the pass totals: exact, so their order does not matter
        __syncthreads();
        const long long* fb = reinterpret_cast<const long long*>(s_bS);
        unsigned long long* acc = reinterpret_cast<unsigned long long*>(a.acc);
        for (int e = tid; e < K * D; e += blockDim.x) {
            const long long v = fb[e];
            if (v != 0) atomicAdd(acc + e, (unsigned long long)v);
        }
        for (int j = tid; j < K; j += blockDim.x) {
            const int c = s_bC[j];
            if (c != 0) atomicAdd(a.accC + j, c);
        }
    } else if (do_bins) {
        __syncthreads();
        T* pS = reinterpret_cast<T*>(a.pS) + (size_t)bid * K * D;
        for (int e = tid; e < K * D; e += blockDim.x) {
            T s = T(0);
            for (int w = 0; w < W; ++w) s += s_bS[(size_t)w * K * D + e];
            pS[e] = s;
        }
        int32_t* pC = a.pCnt + (size_t)bid * K;
        for (int j = tid; j < K; j += blockDim.x) {
            int s = 0;
            for (int w = 0; w < W; ++w) s += s_bC[w * K + j];
            pC[j] = s;
        }
    }

    // ---- last block: fixed-order reduction over blocks and the controller
    __threadfence();
    __syncthreads();
    unsigned int* sflag = reinterpret_cast<unsigned int*>(s_red + 40);
    if (tid == 0) {
        const unsigned int prev = atomicAdd(a.counter, 1u);
        *sflag = (prev == (unsigned)nblk - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (*sflag == 0u) return;
    __threadfence();
    if (a.acc && a.mode == MODE_INIT) {       // the solve's first pass: clear the fixed-point totals
        for (int i = tid; i < K * D; i += blockDim.x) a.acc[i] = 0;
        for (int j = tid; j < K; j += blockDim.x) a.accC[j] = 0;
    }
    double E = 0.0;
    long long ch = 0, rs = 0, bd = 0, sc = 0;
    for (int b = tid; b < nblk; b += blockDim.x) {
        E += __ldcg(a.pE + b);
        ch += __ldcg(a.pNch + b);
        rs += __ldcg(a.pResc + b);
        if (a.pScan) sc += __ldcg(a.pScan + b);
        bd += __ldcg(a.pBad + b);
    }
    E = block_sum_d(E, s_red);
    ch = block_sum_ll(ch, s_red);
    rs = block_sum_ll(rs, s_red);
    sc = block_sum_ll(sc, s_red);
    bd = block_sum_ll(bd, s_red);
    if (ham)
        for (int i = tid; i < K * D; i += blockDim.x) a.hlast[i] = reinterpret_cast<const float*>(s_c)[i];
    if (tid == 0) {
        *a.counter = 0u;
        if (a.mode == MODE_STANDALONE) {
            if (a.out_nch) *a.out_nch = ch;
            if (a.out_E) *a.out_E = E;
        } else {
            st->rescored += rs;
            st->scanned += sc;
            if (fx) st->fx_s = fx_s;
            if (a.mode == MODE_EPI) {
                st->E_final = E;
            } else if (a.mode == MODE_INIT) {
                st->passes += 1;
                st->E_trial = E;
                if (bd) st->status = KM_ENONFINITE;       // the first loop pass stops the solve
            } else {
                if (a.mode == MODE_TRIAL)
                    controller_trial(st, E, ch, a.thr, a.lloyd_only, a.fixed_m, a.eps1, a.eps2, a.m_max, a.max_iter);
                else
                    controller_revert(st, E, ch, a.thr);
                // the kernel that ends the solve also ends the graph's while loop; the TRIAL pass
                // also decides whether the REVERT pass runs at all
                if (st->done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
                if (a.mode == MODE_TRIAL && a.use_cond_rev)
                    cudaGraphSetConditional(a.cond_rev, (st->revert && !st->done) ? 1u : 0u);
            }
        }
    }
    // the safeguard fired: the REVERT pass sums into cleared totals
    if (fx && a.mode == MODE_TRIAL) {
        __syncthreads();
        if (st->revert && !st->done) {
            for (int i = tid; i < K * D; i += blockDim.x) a.acc[i] = 0;
            for (int j = tid; j < K; j += blockDim.x) a.accC[j] = 0;
        }
    }
    // the safeguard fired: the REVERT pass's bound inputs (drift from C^t, just saved as the last
    // centroids, to C_AU), computed here instead of by a launch of their own
    if constexpr (F32) {
        if (ham && a.mode == MODE_TRIAL) {
            __syncthreads();
            if (st->revert && !st->done) hprep_body<D>(a, MODE_REVERT, reinterpret_cast<float*>(s_red));
        }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(LOWD_THREADS, MinBlocks<T, D>::value) k_pass_lowd(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    pass_body<T, D>(a, blockIdx.x, gridDim.x, smem);
}

// Resident blocks per SM of the assignment-only FP32 pass: without the bins and bounds code the
// scan fits 64 registers for d <= 3, so four blocks (32 warps) hide more latency; d = 7, 8 keep
// their registers at two blocks (three spill here).
template <typename T, int D>
struct AoBlocks {
    static constexpr int value = !std::is_same<T, float>::value ? MinBlocks<T, D>::value
                                 : D <= 3                        ? 4
                                 : D <= 6                        ? 3
                                                                 : 2;
};

template <typename T, int D>
__global__ void __launch_bounds__(LOWD_THREADS, AoBlocks<T, D>::value) k_pass_lowd_ao(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    pass_body<T, D, 0, true>(a, blockIdx.x, gridDim.x, smem);
}

// Persistent batched pass: each block takes work items (instance, block of that instance) in
// turn; an item does what that block of the instance's own launch would do (same rows, same
// partial slot, the instance's last item runs its reduction and controller).  No item waits for
// another, so any grid size is safe.
template <typename T, int D, int RV = 0>
__global__ void __launch_bounds__(LOWD_THREADS, MinBlocks<T, D>::value) k_pass_lowd_batch(BatchPass b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const int2 w = b.items[it];
        PassArgs a = b.args[w.x];
        a.mode = b.mode;
        a.flags = b.flags;
        a.use_cond = 0;
        pass_body<T, D, RV>(a, w.y, a.nblk, smem);
        __syncthreads();
    }
}

// Largest dynamic shared memory a kernel may request: the per-block limit minus its static part.
template <typename F>
int dyn_smem_limit(F kern)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return LOWD_SMEM_MAX;
    return LOWD_SMEM_MAX - (int)fa.sharedSizeBytes;
}

template <typename T, int D>
cudaError_t launch_one(const PassArgs& a, int nb, size_t smem, cudaStream_t s)
{
    auto kern = k_pass_lowd<T, D>;
    static bool attr_set = false;
    if (!attr_set || smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<nb, LOWD_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int RV = 0>
cudaError_t launch_batch_one(const BatchPass& b, int grid, size_t smem, cudaStream_t s)
{
    auto kern = k_pass_lowd_batch<T, D, RV>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<grid, LOWD_THREADS, smem, s>>>(b);
    return cudaGetLastError();
}

template <typename T, int D>
cudaError_t launch_one_ao(const PassArgs& a, int nb, size_t smem, cudaStream_t s)
{
    auto kern = k_pass_lowd_ao<T, D>;
    static bool attr_set = false;
    if (!attr_set || smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<nb, LOWD_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D>
int pass_occ_ao(size_t smem)
{
    int n = 0;
    auto kern = k_pass_lowd_ao<T, D>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern)) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, LOWD_THREADS, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <typename T, int D>
int pass_occ(size_t smem)
{
    int n = 0;
    auto kern = k_pass_lowd<T, D>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern)) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, LOWD_THREADS, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

template <typename T, int D, int RV = 0>
int batch_occ(size_t smem)
{
    int n = 0;
    auto kern = k_pass_lowd_batch<T, D, RV>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_limit(kern)) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, LOWD_THREADS, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

}  // namespace km
