// Update step finalisation, Anderson least squares and the accelerated iterate (sm_103a).
//
// k_fin  : fixed-order reduction of the per-block residual sums and counts of a pass into the
//          update step (Eq. 4) written as G(C) = C + F, F_j = (1/N_j) sum_{rho_i=j}(x_i - c_j)
//          (F_j = 0 for an empty cluster, which keeps its centroid).  In the solver it also
//          forms dF = F^t - F^{t-1} and dG = G^t - G^{t-1} (Eq. 7 / Eq. 8 differences) into the
//          history rings and the new row of the FP64 Gram matrix of the dF columns plus the
//          right-hand side <dF_j, F^t> (the "m inner products between (Kd)-dimensional
//          vectors" of Section 2.1).  The last block solves the m_t x m_t least-squares system
//          through the Cholesky factor of the Gram matrix (= the R factor of the QR of dF),
//          dropping columns from the first with R_kk <= rank_tol * R_00 on, and closes the
//          iteration of Algorithm 1.
// k_mix  : C^{t+1} = G^t - sum_j theta_j dG_j (Eq. 8 with Algorithm 1's sign) in FP64 and the
//          FP32 packing of C^{t+1} and G^t for the next assignment passes; the only place that
//          ends the graph's while loop.
// k_prep : once per solve: origin, C^0, packing, controller state.
// k_epi  : once per solve: result centroids, assignment and info.
#include "km_internal.cuh"

namespace km {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Solve the LS problem of Eq. 7 from the Gram matrix: columns a = 0..mt-1 are ring slots
// slot[a] (a = 0 newest).  Cholesky M = L L^T with column truncation; returns the rank.
__device__ int ls_from_gram(const SolveState* st, const int* slot, int mt, double rank_tol,
                            double* theta)
{
    double Lm[MMAX][MMAX];
    double y[MMAX];
    int rank = 0;
    double l00 = 0.0;
    for (int k = 0; k < mt; ++k) {
        double piv = st->gram[slot[k] * MMAX + slot[k]];
        for (int i = 0; i < k; ++i) piv -= Lm[k][i] * Lm[k][i];
        const double lkk = piv > 0.0 ? sqrt(piv) : 0.0;
        if (k == 0) l00 = lkk;
        if (l00 == 0.0 || lkk <= rank_tol * l00) break;
        Lm[k][k] = lkk;
        for (int r = k + 1; r < mt; ++r) {
            double v = st->gram[slot[r] * MMAX + slot[k]];
            for (int i = 0; i < k; ++i) v -= Lm[r][i] * Lm[k][i];
            Lm[r][k] = v / lkk;
        }
        rank = k + 1;
    }
    for (int k = 0; k < rank; ++k) {            // L y = b
        double v = st->bvec[slot[k]];
        for (int i = 0; i < k; ++i) v -= Lm[k][i] * y[i];
        y[k] = v / Lm[k][k];
    }
    for (int k = rank - 1; k >= 0; --k) {       // L^T theta = y
        double v = y[k];
        for (int i = k + 1; i < rank; ++i) v -= Lm[i][k] * theta[i];
        theta[k] = v / Lm[k][k];
    }
    for (int k = rank; k < MMAX; ++k) theta[k] = 0.0;
    return rank;
}

__global__ void __launch_bounds__(FIN_THREADS) k_fin(FinArgs a)
{
    SolveState* st = a.st;
    const bool solver = a.mode != MODE_STANDALONE;
    if (solver && st->done) return;
    const int tid = threadIdx.x;
    const int K = a.K, d = a.d, nb = a.nb;
    const int j0 = blockIdx.x * a.KB;
    const int kb = min(a.KB, K - j0);
    const int E = kb * (d + 1);
    int split = FIN_THREADS / max(E, 1);
    split = split < 1 ? 1 : (split > 8 ? 8 : split);

    extern __shared__ __align__(16) unsigned char smem[];
    double* s_tot = reinterpret_cast<double*>(smem);             // [E]
    double* s_dfn = s_tot + E;                                    // [kb*d]
    double* s_F = s_dfn + (size_t)kb * d;                         // [kb*d]
    double* s_part = s_F + (size_t)kb * d;                        // [FIN_THREADS] (split > 1)
    double* s_red = s_part + FIN_THREADS;                         // [2*MMAX*8]

    // ---- phase 1/2: sums over partial blocks in a fixed order
    if (split > 1) {
        for (int p = tid; p < E * split; p += blockDim.x) {
            const int e = p / split, s = p % split;
            double acc = 0.0;
            if (e < kb * d) {
                const size_t off = (size_t)j0 * d + e;
                if (a.part_f64) {
                    const double* pS = reinterpret_cast<const double*>(a.pS);
                    for (int b = s; b < nb; b += split) acc += pS[(size_t)b * K * d + off];
                } else {
                    const float* pS = reinterpret_cast<const float*>(a.pS);
                    for (int b = s; b < nb; b += split) acc += (double)pS[(size_t)b * K * d + off];
                }
            } else {
                const int j = j0 + (e - kb * d);
                long long c = 0;
                for (int b = s; b < nb; b += split) c += a.pCnt[(size_t)b * K + j];
                acc = (double)c;
            }
            s_part[p] = acc;
        }
        __syncthreads();
        for (int e = tid; e < E; e += blockDim.x) {
            double v = 0.0;
            for (int s = 0; s < split; ++s) v += s_part[e * split + s];
            s_tot[e] = v;
        }
    } else {
        for (int e = tid; e < E; e += blockDim.x) {
            double acc = 0.0;
            if (e < kb * d) {
                const size_t off = (size_t)j0 * d + e;
                if (a.part_f64) {
                    const double* pS = reinterpret_cast<const double*>(a.pS);
                    for (int b = 0; b < nb; ++b) acc += pS[(size_t)b * K * d + off];
                } else {
                    const float* pS = reinterpret_cast<const float*>(a.pS);
                    for (int b = 0; b < nb; ++b) acc += (double)pS[(size_t)b * K * d + off];
                }
            } else {
                const int j = j0 + (e - kb * d);
                long long c = 0;
                for (int b = 0; b < nb; ++b) c += a.pCnt[(size_t)b * K + j];
                acc = (double)c;
            }
            s_tot[e] = acc;
        }
    }
    __syncthreads();

    // ---- phase 3: per element
    if (!solver) {
        for (int e = tid; e < kb * d; e += blockDim.x) {
            const size_t i = (size_t)j0 * d + e;
            const double Nj = s_tot[kb * d + e / d];
            if (a.out_f64) {
                const double cr = reinterpret_cast<const double*>(a.C_ref)[i];
                reinterpret_cast<double*>(a.C_out)[i] = Nj > 0.0 ? cr + s_tot[e] / Nj : cr;
            } else {
                const double cr = (double)reinterpret_cast<const float*>(a.C_ref)[i];
                reinterpret_cast<float*>(a.C_out)[i] = (float)(Nj > 0.0 ? cr + s_tot[e] / Nj : cr);
            }
        }
        if (a.counts)
            for (int e = tid; e < kb; e += blockDim.x) a.counts[j0 + e] = (int64_t)s_tot[kb * d + e];
        return;
    }

    const bool init = a.mode == MODE_INIT;
    const bool ring = !init && a.m_max > 0 && !a.lloyd_only;
    const int m_max = a.m_max;
    const int head = st->ring_head, count = st->ring_count;
    const int hnew = ring ? (head + 1) % m_max : 0;
    const int nold = ring ? min(count, m_max - 1) : 0;
    const double* Ct = st->revert ? a.CAU : a.C64;
    for (int e = tid; e < kb * d; e += blockDim.x) {
        const size_t i = (size_t)j0 * d + e;
        const double Nj = s_tot[kb * d + e / d];
        const double F = Nj > 0.0 ? s_tot[e] / Nj : 0.0;
        const double c = Ct[i];
        const double G = c + F;
        if (ring) {
            const size_t n = (size_t)K * d;
            const double dfn = F - a.Fprev[i];
            const double dgn = G - a.CAU[i];
            a.dF[(size_t)hnew * n + i] = dfn;
            a.dG[(size_t)hnew * n + i] = dgn;
            s_dfn[e] = dfn;
            s_F[e] = F;
        }
        a.Fprev[i] = F;
        a.CAU[i] = G;
    }
    if (!ring) {
        // no least squares: a plain Lloyd step; still close the iteration in the last block
    }
    __syncthreads();

    // ---- dot partials: age 0 = the new column, age s >= 1 = slot (head - s + 1)
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nage = ring ? nold + 1 : 0;
    if (ring) {
        const size_t n = (size_t)K * d;
        for (int s = 0; s < nage; ++s) {
            const int q = s == 0 ? hnew : (head - (s - 1) + m_max) % m_max;
            double gv = 0.0, bv = 0.0;
            for (int e = tid; e < kb * d; e += blockDim.x) {
                const size_t i = (size_t)j0 * d + e;
                const double col = s == 0 ? s_dfn[e] : a.dF[(size_t)q * n + i];
                gv += s_dfn[e] * col;
                bv += col * s_F[e];
            }
            gv = warp_sum(gv);
            bv = warp_sum(bv);
            if (lane == 0) {
                s_red[(2 * s) * 8 + warp] = gv;
                s_red[(2 * s + 1) * 8 + warp] = bv;
            }
        }
        __syncthreads();
        for (int v = tid; v < 2 * nage; v += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < nw; ++w) acc += s_red[v * 8 + w];
            a.pDots[(size_t)blockIdx.x * DOTS + v] = acc;
        }
    }

    // ---- last block: Gram update, least squares, end of iteration
    __threadfence();
    __syncthreads();
    __shared__ unsigned int s_last;
    if (tid == 0) s_last = (atomicAdd(&st->ctr_fin, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (ring) {
        for (int v = tid; v < 2 * nage; v += blockDim.x) {
            double acc = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) acc += __ldcg(a.pDots + (size_t)b * DOTS + v);
            s_red[v] = acc;
        }
        __syncthreads();
    }
    if (tid != 0) return;
    st->ctr_fin = 0u;
    if (init) {
        st->t = 1;
        st->cur = 1;
        st->revert = 0;
        return;
    }
    int rank = 0, mt = 0;
    if (ring) {
        st->gram[hnew * MMAX + hnew] = s_red[0];
        st->bvec[hnew] = s_red[1];
        for (int s = 1; s < nage; ++s) {
            const int q = (head - (s - 1) + m_max) % m_max;
            st->gram[hnew * MMAX + q] = s_red[2 * s];
            st->gram[q * MMAX + hnew] = s_red[2 * s];
            st->bvec[q] = s_red[2 * s + 1];
        }
        st->ring_head = hnew;
        st->ring_count = min(count + 1, m_max);
        mt = min(min(st->m, st->t), st->ring_count);
        int slot[MMAX];
        for (int k = 0; k < mt; ++k) slot[k] = (hnew - k + m_max) % m_max;
        double th[MMAX];
        rank = mt > 0 ? ls_from_gram(st, slot, mt, a.rank_tol, th) : 0;
        for (int k = 0; k < MMAX; ++k) st->theta[k] = k < rank ? th[k] : 0.0;
    }
    st->m_t = mt;
    st->rank = rank;
    st->from_lloyd = rank == 0;
    st->E_prev2 = st->E_prev;
    st->E_prev = st->E_cur;
    if (st->t >= a.max_iter) {
        st->done = 1;
        st->converged = 0;
        st->final_src = 1;          // (P^t, G^t)
    } else {
        st->t += 1;
        st->cur ^= 1;
        st->revert = 0;
    }
}

__global__ void __launch_bounds__(256) k_mix(MixArgs a, int use_cond, cudaGraphConditionalHandle cond,
                                             int max_iter)
{
    SolveState* st = a.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the single place that ends the graph's loop: done, or a hard iteration guard
        int stop = st->done;
        st->pad += 1;                                   // body executions (guard)
        if (!stop && (int)st->pad > max_iter + 2) {
            st->status = KM_ETIMEOUT;
            st->done = 1;
            stop = 1;
        }
        if (stop && use_cond) cudaGraphSetConditional(cond, 0);
    }
    if (st->done) return;
    const int K = a.K, d = a.d;
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= K) return;
    const size_t n = (size_t)K * d;
    const int rank = a.mode == MODE_INIT ? 0 : st->rank;
    const int head = st->ring_head, m_max = a.m_max;
    double th[MMAX];
    int sl[MMAX];
    for (int k = 0; k < rank; ++k) {
        th[k] = st->theta[k];
        sl[k] = (head - k + m_max) % m_max;
    }
    double nrm0 = 0.0, nrm1 = 0.0;
    for (int k = lane; k < d; k += 32) {
        const size_t i = (size_t)j * d + k;
        const double g = a.CAU[i];
        double c = g;
        for (int q = 0; q < rank; ++q) c -= th[q] * a.dG[(size_t)sl[q] * n + i];
        a.C64[i] = c;
        if (a.fp32_path) {
            const double o = (double)a.origin[k];
            const float c0 = (float)(c - o), c1 = (float)(g - o);
            a.c32[0][i] = (float)c;
            a.c32[1][i] = (float)g;
            a.cpk[0][(size_t)j * a.DP + k] = -2.f * c0;
            a.cpk[1][(size_t)j * a.DP + k] = -2.f * c1;
            nrm0 += (double)c0 * (double)c0;
            nrm1 += (double)c1 * (double)c1;
        }
    }
    if (a.fp32_path) {
        nrm0 = warp_sum(nrm0);
        nrm1 = warp_sum(nrm1);
        if (lane == 0) {
            a.cpk[0][(size_t)j * a.DP + d] = (float)nrm0;
            a.cpk[1][(size_t)j * a.DP + d] = (float)nrm1;
        }
    }
}

template <typename T>
__global__ void k_prep(const T* C0, int K, int d, int Kpad, int DP, int fp32_path, double* C64,
                       float* origin, float* cpk0, float* cpk1, float* c32_0, SolveState* st,
                       int m_init, int m_max)
{
    const int tid = threadIdx.x;
    __shared__ double s_o[64];
    // origin o = mean of the initial centroids (FP64, ascending j), rounded to FP32
    if (fp32_path) {
        for (int k = tid; k < d; k += blockDim.x) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += (double)C0[(size_t)j * d + k];
            origin[k] = (float)(s / K);
        }
    }
    __syncthreads();
    const size_t n = (size_t)K * d;
    for (size_t i = tid; i < n; i += blockDim.x) C64[i] = (double)C0[i];
    if (fp32_path) {
        for (size_t i = tid; i < (size_t)Kpad * DP; i += blockDim.x) {
            const int j = (int)(i / DP), k = (int)(i % DP);
            const float v = (j >= K && k == d) ? __int_as_float(0x7f800000) : 0.f;
            cpk0[i] = v;
            cpk1[i] = v;
        }
        __syncthreads();
        for (int j = tid; j < K; j += blockDim.x) {
            double nrm = 0.0;
            for (int k = 0; k < d; ++k) {
                const double c = (double)C0[(size_t)j * d + k];
                const float cc = (float)(c - (double)origin[k]);
                c32_0[(size_t)j * d + k] = (float)c;
                cpk0[(size_t)j * DP + k] = -2.f * cc;
                nrm += (double)cc * (double)cc;
            }
            cpk0[(size_t)j * DP + d] = (float)nrm;
        }
    }
    if (tid == 0) {
        SolveState s;
        memset(&s, 0, sizeof(s));
        s.m = m_init < m_max ? m_init : m_max;
        if (s.m < 0) s.m = 0;
        s.from_lloyd = 1;
        s.E_prev = s.E_prev2 = __longlong_as_double(0x7ff0000000000000LL);
        s.ring_head = -1 + (m_max > 0 ? m_max : 1);      // first insert goes to slot 0
        s.ring_count = 0;
        s.status = KM_OK;
        *st = s;
    }
    (void)s_o;
}

struct DevInfo {
    int iters, accepted, rejected, passes, converged, m_final, status, pad;
    double E;
    long long rescored;
};

template <typename T>
__global__ void k_epi(const SolveState* st, const double* C64, const double* CAU, T* C_out, size_t n,
                      const int32_t* rhoA, const int32_t* rhoB, int32_t* rho_out, int64_t N, DevInfo* info)
{
    const double* src = st->final_src ? CAU : C64;
    const int32_t* rho = st->cur ? rhoB : rhoA;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, T_ = (size_t)gridDim.x * blockDim.x;
    for (size_t i = tid; i < n; i += T_) C_out[i] = (T)src[i];
    for (size_t i = tid; i < (size_t)N; i += T_) rho_out[i] = rho[i];
    if (tid == 0) {
        DevInfo f;
        f.iters = st->t;
        f.accepted = st->accepted;
        f.rejected = st->rejected;
        f.passes = st->passes;
        f.converged = st->converged;
        f.m_final = st->m;
        f.status = st->status;
        f.pad = 0;
        f.E = st->E_final;
        f.rescored = st->rescored;
        *info = f;
    }
}

}  // namespace

int fin_blocks(int K, int d, int* KB)
{
    int kb = 32 / (d + 1);
    if (kb < 1) kb = 1;
    *KB = kb;
    return (K + kb - 1) / kb;
}

cudaError_t launch_fin(const FinArgs& a, int nblocks, cudaStream_t s)
{
    const int E = a.KB * (a.d + 1);
    const size_t smem = sizeof(double) * ((size_t)E + 2 * (size_t)a.KB * a.d + FIN_THREADS + 2 * MMAX * 8);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fin<<<nblocks, FIN_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mix_full(const MixArgs& a, int use_cond, cudaGraphConditionalHandle cond, int max_iter,
                            cudaStream_t s)
{
    const int warps = a.K;
    const int blocks = (warps * 32 + 255) / 256;
    k_mix<<<blocks, 256, 0, s>>>(a, use_cond, cond, max_iter);
    return cudaGetLastError();
}

cudaError_t launch_prep(const void* C0, bool f64, int K, int d, int Kpad, int DP, double* C64,
                        float* origin, float* cpk0, float* cpk1, float* c32_0, SolveState* st, int m_init,
                        int m_max, cudaStream_t s)
{
    if (f64)
        k_prep<double><<<1, 1024, 0, s>>>(reinterpret_cast<const double*>(C0), K, d, Kpad, DP, 0, C64, origin,
                                          cpk0, cpk1, c32_0, st, m_init, m_max);
    else
        k_prep<float><<<1, 1024, 0, s>>>(reinterpret_cast<const float*>(C0), K, d, Kpad, DP, 1, C64, origin,
                                         cpk0, cpk1, c32_0, st, m_init, m_max);
    return cudaGetLastError();
}

cudaError_t launch_epi(bool f64, const SolveState* st, const double* C64, const double* CAU, void* C_out,
                       size_t n, const int32_t* rhoA, const int32_t* rhoB, int32_t* rho_out, int64_t N,
                       void* info, cudaStream_t s)
{
    const int blocks = 152;
    if (f64)
        k_epi<double><<<blocks, 256, 0, s>>>(st, C64, CAU, reinterpret_cast<double*>(C_out), n, rhoA, rhoB,
                                             rho_out, N, reinterpret_cast<DevInfo*>(info));
    else
        k_epi<float><<<blocks, 256, 0, s>>>(st, C64, CAU, reinterpret_cast<float*>(C_out), n, rhoA, rhoB,
                                            rho_out, N, reinterpret_cast<DevInfo*>(info));
    return cudaGetLastError();
}

size_t devinfo_bytes() { return sizeof(DevInfo); }

}  // namespace km
