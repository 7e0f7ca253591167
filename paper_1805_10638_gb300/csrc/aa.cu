// Update step finalisation, Anderson least squares and the accelerated iterate (sm_103a).
//
// k_fin  : fixed-order reduction of the per-block residual sums and counts of a pass into the
//          update step (Eq. 4) written as G(C) = C + F, F_j = (1/N_j) sum_{rho_i=j}(x_i - c_j)
//          (F_j = 0 for an empty cluster, which keeps its centroid).  In the solver it also
//          forms dF = F^t - F^{t-1} and dG = G^t - G^{t-1} (the differences of Eq. 7 / Eq. 8)
//          into the history rings, and the new row of the FP64 Gram matrix of the dF columns
//          plus the right-hand side <dF_j, F^t> (m inner products of length K*d, the per-
//          iteration cost Section 2.1 counts).  The last block solves the m_t x m_t least-squares problem
//          through the Cholesky factor of the Gram matrix (= the R factor of the QR of dF),
//          dropping columns from the first with R_kk <= rank_tol * R_00 on, closes the iteration
//          of Algorithm 1 and, when K*d is small, also forms the accelerated iterate.
// k_mix  : C^{t+1} = G^t - sum_j theta_j dG_j (Eq. 8 with Algorithm 1's sign) in FP64 and the
//          FP32 packing of C^{t+1} and G^t for the next assignment passes (large K*d).
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

// Least squares of Eq. 7 from the Gram matrix, by one warp: columns a = 0..mt-1 are ring slots
// (hnew - a) mod m_max (a = 0 newest).  Right-looking Cholesky M = L L^T in shared memory, lane r
// owning row r, with 1/L_kk from rsqrt (no divisions).  The Cholesky factor of the Gram matrix is
// the R of the QR of dF, but its small pivots carry an error of about u (L_00 / L_kk)^2 relative
// (the Gram matrix squares the condition number).  So the factor is only trusted while every
// pivot ratio L_kk / L_00 stays above cert_tol: a column from the first with L_kk <= rank_tol *
// L_00 on is then dropped as the QR would drop it.  A pivot ratio at or below cert_tol (cert_tol >
// 0) stops the factorisation with *uncert = 1 and the caller solves by Householder QR instead
// (ls_qr_block).  cert_tol = 0 trusts every pivot (the Gram route alone).  Forward and back
// substitution give theta.  Returns the rank (in every lane); theta[0..MMAX) in shared memory.
__device__ __forceinline__ int ls_warp(const SolveState* st, int hnew, int m_max, int mt, double rank_tol,
                                       double cert_tol, int* uncert, double* sM, double* sInv, double* sV)
{
    const int lane = threadIdx.x & 31;
    const int sr = lane < mt ? (hnew - lane + m_max) % m_max : 0;
    for (int c = 0; c < mt; ++c) {
        const int sc = (hnew - c + m_max) % m_max;
        if (lane < mt) sM[lane * MMAX + c] = st->gram[sr * MMAX + sc];
    }
    sV[lane] = lane < mt ? st->bvec[sr] : 0.0;
    __syncwarp();
    int rank = 0;
    double l00 = 0.0;
    for (int k = 0; k < mt; ++k) {
        const double piv = sM[k * MMAX + k];
        const double r = piv > 0.0 ? rsqrt(piv) : 0.0;
        const double lkk = piv * r;
        if (k == 0) l00 = lkk;
        if (l00 == 0.0) break;
        if (cert_tol > 0.0 && !(lkk > cert_tol * l00)) {
            *uncert = 1;
            break;
        }
        if (!(lkk > rank_tol * l00)) break;
        __syncwarp();
        if (lane > k && lane < mt) sM[lane * MMAX + k] *= r;
        if (lane == k) {
            sM[k * MMAX + k] = lkk;
            sInv[k] = r;
        }
        __syncwarp();
        if (lane > k && lane < mt) {
            const double lrk = sM[lane * MMAX + k];
            for (int j = k + 1; j <= lane; ++j) sM[lane * MMAX + j] -= lrk * sM[j * MMAX + k];
        }
        __syncwarp();
        rank = k + 1;
    }
    for (int k = 0; k < rank; ++k) {               // L y = b
        const double yk = sV[k] * sInv[k];
        __syncwarp();
        if (lane == k) sV[k] = yk;
        if (lane > k && lane < rank) sV[lane] -= sM[lane * MMAX + k] * yk;
        __syncwarp();
    }
    for (int k = rank - 1; k >= 0; --k) {          // L^T theta = y
        const double tk = sV[k] * sInv[k];
        __syncwarp();
        if (lane == k) sV[k] = tk;
        if (lane < k) sV[lane] -= sM[k * MMAX + lane] * tk;
        __syncwarp();
    }
    if (lane >= rank) sV[lane] = 0.0;
    __syncwarp();
    return rank;
}

// The same solve with the Gram rows in registers (lane r holds row r, MB >= mt columns), so that
// the rank-1 updates of a column are independent FMAs instead of a chain through shared memory.
// Every FP64 operation and its order match ls_warp, so the results are bitwise the same.
template <int MB>
__device__ __forceinline__ int ls_warp_reg(const SolveState* st, int hnew, int m_max, int mt, double rank_tol,
                                           double cert_tol, int* uncert, double* sM, double* sV)
{
    const int lane = threadIdx.x & 31;
    const int sr = lane < mt ? (hnew >= lane ? hnew - lane : hnew - lane + m_max) : 0;   // mt <= m_max
    double m[MB];
#pragma unroll
    for (int c = 0; c < MB; ++c) {
        const int sc = hnew >= c ? hnew - c : hnew - c + m_max;
        m[c] = (lane < mt && c < mt) ? st->gram[sr * MMAX + sc] : 0.0;
    }
    double v = lane < mt ? st->bvec[sr] : 0.0;
    double inv[MB];
    int rank = 0;
    double l00 = 0.0;
    bool go = true;
#pragma unroll
    for (int k = 0; k < MB; ++k) {
        inv[k] = 0.0;
        if (go && k < mt) {
            const double piv = __shfl_sync(FULL, m[k], k);
            const double r = piv > 0.0 ? rsqrt(piv) : 0.0;
            const double lkk = piv * r;
            if (k == 0) l00 = lkk;
            if (l00 != 0.0 && cert_tol > 0.0 && !(lkk > cert_tol * l00)) {
                *uncert = 1;
                go = false;
            } else if (l00 == 0.0 || !(lkk > rank_tol * l00)) {
                go = false;
            } else {
                if (lane > k && lane < mt) m[k] *= r;
                if (lane == k) m[k] = lkk;
                inv[k] = r;
#pragma unroll
                for (int j = k + 1; j < MB; ++j) {
                    if (j >= mt) break;          // uniform: no FP64 issue for columns past the history
                    const double ljk = __shfl_sync(FULL, m[k], j);
                    if (lane >= j && lane < mt) m[j] -= m[k] * ljk;
                }
                rank = k + 1;
                // L y = b, step k, as soon as column k is final (off the pivot chain)
                const double yk = __shfl_sync(FULL, v, k) * inv[k];
                if (lane == k) v = yk;
                if (lane > k && lane < mt) v -= m[k] * yk;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < MB; ++c) sM[lane * MMAX + c] = m[c];
    __syncwarp();
    double colL[MB];                           // colL[k] = L[k][lane]
#pragma unroll
    for (int k = 0; k < MB; ++k) colL[k] = k < 32 ? sM[k * MMAX + lane] : 0.0;
#pragma unroll
    for (int k = MB - 1; k >= 0; --k) {        // L^T theta = y
        if (k < rank) {
            const double tk = __shfl_sync(FULL, v, k) * inv[k];
            if (lane == k) v = tk;
            if (lane < k) v -= colL[k] * tk;
        }
    }
    sV[lane] = lane < rank ? v : 0.0;
    __syncwarp();
    return rank;
}

// Least squares of Eq. 7 by Householder QR of [dF | f], by one whole block: the path taken when the
// Gram route cannot certify the factor (ls_warp / ls_warp_reg) and the one the QR-only mode
// always takes.  Column q < mt of the n x (mt + 1) working matrix W (global scratch, column-major)
// is the ring slot sl[q] of dF (q = 0 newest); column mt is f = F^t.  Step k reflects rows k..n-1
// with H_k = I - 2 v v^T / (v^T v), v = a_k - alpha e_k, alpha = -sign(a_kk) ||a_k||, R_kk = alpha;
// the reflector is applied to the later columns and to f, so f's column ends as Q^T f.  As in the
// oracle, the first column with |R_kk| <= rank_tol |R_00| (or R_00 = 0) and every later (older) one
// are dropped (theta = 0).  The dot products of a step are summed per thread over fixed rows, then
// over lanes and warps in a fixed order, so the result is the same on every run.  Cost: about
// n (mt + 1)(mt + 2) FP64 FMAs on one SM; on data where the Gram route certifies the factor
// (every pivot ratio above cert_tol) it never runs.  Returns the rank; th[0..MMAX) in shared memory.
__device__ __noinline__ int ls_qr_block(const double* dF, const int* sl, int mt, const double* f, size_t n,
                                        double rank_tol, double* W, double* th)
{
    constexpr int CW = 8;                                  // columns per sweep of the dot products
    __shared__ double s_R[MMAX * (MMAX + 1)];             // row k: R_kj (j < mt) and (Q^T f)_k (j = mt)
    __shared__ double s_red[(FIN_THREADS / 32) * CW];
    __shared__ double s_dot[MMAX + 1];
    __shared__ double s_w[MMAX + 1];
    __shared__ double s_r00;
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nc = mt + 1;
    for (int q = 0; q < nc; ++q) {
        const double* src = q < mt ? dF + (size_t)sl[q] * n : f;
        for (size_t i = tid; i < n; i += blockDim.x) W[(size_t)q * n + i] = __ldcg(src + i);
    }
    __syncthreads();
    const int steps = (size_t)mt < n ? mt : (int)n;
    int rank = 0;
    for (int k = 0; k < steps; ++k) {
        const double* ak = W + (size_t)k * n;
        for (int j0 = k; j0 < nc; j0 += CW) {              // s_dot[j] = sum_{i >= k} a_ik a_ij, j = k..mt
            double acc[CW];
#pragma unroll
            for (int c = 0; c < CW; ++c) acc[c] = 0.0;
            for (size_t i = (size_t)k + tid; i < n; i += blockDim.x) {
                const double v = ak[i];
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    if (j0 + c < nc) acc[c] = fma(v, W[(size_t)(j0 + c) * n + i], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                const double v = warp_sum(acc[c]);
                if (lane == 0) s_red[warp * CW + c] = v;
            }
            __syncthreads();
            if (tid < CW && j0 + tid < nc) {
                double v = 0.0;
                for (int w = 0; w < nw; ++w) v += s_red[w * CW + tid];
                s_dot[j0 + tid] = v;
            }
            __syncthreads();
        }
        if (tid == 0) {
            const double nrm2 = s_dot[k], akk = ak[k];
            const double nrm = sqrt(nrm2);
            const double alpha = akk >= 0.0 ? -nrm : nrm;
            const double rkk = fabs(alpha);
            if (k == 0) s_r00 = rkk;
            const int stop = s_r00 == 0.0 || rkk <= rank_tol * s_r00;
            if (!stop) {
                const double vk = akk - alpha;
                const double vtv = 2.0 * (nrm2 - alpha * akk);     // ||a_k - alpha e_k||^2
                s_R[k * (MMAX + 1) + k] = alpha;
                for (int j = k + 1; j < nc; ++j) {
                    const double ajk = W[(size_t)j * n + k];
                    const double w = 2.0 * (s_dot[j] - alpha * ajk) / vtv;   // 2 v.a_j / v.v
                    s_w[j] = w;
                    s_R[k * (MMAX + 1) + j] = ajk - w * vk;
                }
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        rank = k + 1;
        for (size_t i = (size_t)k + 1 + tid; i < n; i += blockDim.x) {   // rows below k: v_i = a_ik
            const double v = ak[i];
            for (int j = k + 1; j < nc; ++j) W[(size_t)j * n + i] = fma(-s_w[j], v, W[(size_t)j * n + i]);
        }
        __syncthreads();
    }
    if (tid == 0) {                                        // R[0:rank, 0:rank] theta = (Q^T f)[0:rank]
        for (int k = rank - 1; k >= 0; --k) {
            double v = s_R[k * (MMAX + 1) + mt];
            for (int j = k + 1; j < rank; ++j) v -= s_R[k * (MMAX + 1) + j] * th[j];
            th[k] = v / s_R[k * (MMAX + 1) + k];
        }
    }
    __syncthreads();
    if (tid >= rank && tid < MMAX) th[tid] = 0.0;
    __syncthreads();
    return rank;
}

// C^{t+1}_j = G^t_j - sum_q theta_q dG_q,j for one centroid (one warp, lanes over d), written to
// C64, and the FP32 packing of C^{t+1} (set 0) and G^t (set 1).  Reads go through L2 (__ldcg):
// G^t and dG were written by other blocks of the same kernel when called from k_fin.
__device__ void mix_pack_centroid(int j, int K, int d, int DP, int fp32_path, double* C64, const double* CAU,
                                  const double* dG, const double* th, const int* sl, int rank, const float* origin,
                                  float* const* cpk, float* const* c32)
{
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)K * d;
    double nrm0 = 0.0, nrm1 = 0.0;
    for (int k = lane; k < d; k += 32) {
        const size_t i = (size_t)j * d + k;
        const double g = __ldcg(CAU + i);
        double dg[MMAX];
#pragma unroll
        for (int q = 0; q < MMAX; ++q) dg[q] = q < rank ? __ldcg(dG + (size_t)sl[q] * n + i) : 0.0;
        double c = g;
#pragma unroll
        for (int q = 0; q < MMAX; ++q)
            if (q < rank) c -= th[q] * dg[q];
        C64[i] = c;
        if (fp32_path) {
            const double o = (double)origin[k];
            const float c0 = (float)(c - o), c1 = (float)(g - o);
            c32[0][i] = (float)c;
            c32[1][i] = (float)g;
            cpk[0][pk_index(j, k, DP)] = -2.f * c0;
            cpk[1][pk_index(j, k, DP)] = -2.f * c1;
            nrm0 += (double)c0 * (double)c0;
            nrm1 += (double)c1 * (double)c1;
        }
    }
    if (fp32_path) {
        nrm0 = warp_sum(nrm0);
        nrm1 = warp_sum(nrm1);
        if (lane == 0) {
            cpk[0][pk_index(j, d, DP)] = (float)nrm0;
            cpk[1][pk_index(j, d, DP)] = (float)nrm1;
        }
    }
}

// sum_{b = b0, b0 + step, ... < nb} p[b * stride] in that order, 16 loads in flight (predicated,
// so a short tail costs no serial round trips).
template <typename V, typename Acc>
__device__ __forceinline__ Acc strided_sum(const V* p, size_t stride, int b0, int nb, int step)
{
    Acc acc = Acc(0);
    for (int b = b0; b < nb; b += 16 * step) {
        V v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int bb = b + u * step;
            v[u] = bb < nb ? p[(size_t)bb * stride] : V(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) acc += (Acc)v[u];
    }
    return acc;
}

// The work of block `bid` of a finalize launch with `nblk` blocks (see k_fin / k_fin_batch).
__device__ __forceinline__ void fin_body(const FinArgs& a, const int bid, const int nblk, unsigned char* smem)
{
    SolveState* st = a.st;
    const bool solver = a.mode != MODE_STANDALONE;
    if (solver && st->done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K, d = a.d, nb = a.nb;
    const int j0 = bid * a.KB;
    const int kb = min(a.KB, K - j0);
    const int E = kb * (d + 1);
    int split = FIN_THREADS / max(E, 1);
    split = split < 1 ? 1 : (split > 32 ? 32 : split);

    double* s_tot = reinterpret_cast<double*>(smem);             // [E]
    double* s_dfn = s_tot + E;                                    // [kb*d]
    double* s_F = s_dfn + (size_t)kb * d;                         // [kb*d]
    double* s_part = s_F + (size_t)kb * d;                        // [2*FIN_THREADS] (>= 2*MMAX*8)
    double* s_red = s_part + 2 * FIN_THREADS;                     // [2*MMAX*8]
    __shared__ double s_M[MMAX * MMAX];
    __shared__ double s_inv[MMAX];
    __shared__ double s_th[MMAX];
    __shared__ int s_sl[MMAX];
    __shared__ int s_rank;
    __shared__ int s_unc;
    __shared__ unsigned int s_last;

    // ---- phase 1/2: sums over the partial blocks in a fixed order.  With split == 1 (E >= the
    // block size) each element goes straight to s_tot; s_part holds only 2*FIN_THREADS entries.
    // FP32 solver passes after the first (d <= FX_MAX_D), and every dense update, sum in 64-bit
    // fixed point (scale 2^fx_s) straight into the totals acc / accC: read once, converted to FP64 once, and
    // cleared for the next pass.  Counts of the other passes are summed as integers.
    // the incremental update (dense solver passes) keeps raw sums of x per cluster instead of the
    // residuals' sums: F = S / N_j - c there
    const bool raw = solver && a.inc && a.part_fx == 2;
    const long long* accp = raw ? a.Spair[st->cur] : a.acc;
    const int32_t* accCp = raw ? a.Npair[st->cur] : a.accC;
    const bool fxp = accp && (a.part_fx == 2 || (a.part_fx == 1 && solver && a.mode != MODE_INIT));
    const int fxs = fxp ? (a.fxs_ptr ? *a.fxs_ptr : st->fx_s) : 0;
    long long* s_ipart = reinterpret_cast<long long*>(s_part);
    const size_t Kd = (size_t)K * d;
    // (e, sp): element e, blocks sp, sp + split, ...; split == 1 writes s_tot directly.  Consecutive
    // threads take consecutive elements of the same partial block (coalesced loads).
    for (int p = tid; p < E * split; p += blockDim.x) {
        const int sp = p / E, e = p - sp * E;
        const bool isum = e >= kb * d || fxp;          // integer sum
        long long is = 0;
        double acc = 0.0;
        if (e < kb * d) {
            const size_t off = (size_t)j0 * d + e;
            if (fxp) is = sp == 0 ? accp[off] : 0;        // the pass's exact total
            else if (a.part_f64) acc = strided_sum<double, double>(reinterpret_cast<const double*>(a.pS) + off, Kd, sp, nb, split);
            else acc = strided_sum<float, double>(reinterpret_cast<const float*>(a.pS) + off, Kd, sp, nb, split);
        } else {
            const int j = j0 + (e - kb * d);
            is = fxp ? (sp == 0 ? (long long)accCp[j] : 0) : strided_sum<int32_t, long long>(a.pCnt + j, (size_t)K, sp, nb, split);
        }
        if (split == 1)
            s_tot[e] = !isum ? acc : (e >= kb * d ? (double)is : ldexp((double)is, -fxs));
        else if (isum)
            s_ipart[e * split + sp] = is;
        else
            s_part[e * split + sp] = acc;
    }
    __syncthreads();
    if (fxp && !raw) {                           // read by this block only: clear for the next pass
        for (int e = tid; e < kb * d; e += blockDim.x) a.acc[(size_t)j0 * d + e] = 0;
        for (int e = tid; e < kb; e += blockDim.x) a.accC[j0 + e] = 0;
    }
    for (int e = tid; split > 1 && e < E; e += blockDim.x) {
        if (e >= kb * d || fxp) {
            long long v = 0;
            for (int sp = 0; sp < split; ++sp) v += s_ipart[e * split + sp];
            s_tot[e] = e >= kb * d ? (double)v : ldexp((double)v, -fxs);
        } else {
            double v = 0.0;
            for (int sp = 0; sp < split; ++sp) v += s_part[e * split + sp];
            s_tot[e] = v;
        }
    }
    __syncthreads();
    // 1/N_j once per centroid
    for (int e = tid; e < kb; e += blockDim.x) {
        const double Nj = s_tot[kb * d + e];
        s_part[e] = Nj > 0.0 ? 1.0 / Nj : 0.0;
    }
    __syncthreads();

    // ---- phase 3: per element
    if (!solver) {
        for (int e = tid; e < kb * d; e += blockDim.x) {
            const size_t i = (size_t)j0 * d + e;
            const double inv = s_part[e / d];
            if (a.out_f64) {
                const double cr = reinterpret_cast<const double*>(a.C_ref)[i];
                reinterpret_cast<double*>(a.C_out)[i] = inv > 0.0 ? cr + s_tot[e] * inv : cr;
            } else {
                const double cr = (double)reinterpret_cast<const float*>(a.C_ref)[i];
                reinterpret_cast<float*>(a.C_out)[i] = (float)(inv > 0.0 ? cr + s_tot[e] * inv : cr);
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
    const size_t n = (size_t)K * d;
    for (int e = tid; e < kb * d; e += blockDim.x) {
        const size_t i = (size_t)j0 * d + e;
        const double c = Ct[i];
        const double inv = s_part[e / d];
        const double F = !raw ? s_tot[e] * inv : (inv > 0.0 ? s_tot[e] * inv - c : 0.0);
        const double G = c + F;
        if (ring) {
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
    __syncthreads();

    // ---- dot partials of this block's elements: age 0 = the new column, age s >= 1 = ring slot
    // (head - s + 1).  Each age gets a group of G = FIN_THREADS / A threads (A = nage rounded up to
    // a power of two); a group's threads take the elements r, r + G, ... and the group is reduced
    // by shuffles within its warp and, when it spans several warps, through shared memory in warp
    // order.  Every product is formed once, and every FP64 instruction does useful work in most
    // lanes: FP64 issue is scarce on this part.
    const int nage = ring ? nold + 1 : 0;
    if (ring) {
        int A = 1;
        while (A < nage) A <<= 1;
        const int G = FIN_THREADS / A;
        const int s = tid / G, r = tid - s * G;
        double g = 0.0, bb = 0.0;
        if (s < nage) {
            const double* col = s == 0 ? s_dfn
                                       : a.dF + (size_t)((head - (s - 1) + m_max) % m_max) * n + (size_t)j0 * d;
#pragma unroll 4
            for (int e = r; e < kb * d; e += G) {
                const double c = col[e];
                g = fma(s_dfn[e], c, g);
                bb = fma(c, s_F[e], bb);
            }
        }
        const int Wg = G < 32 ? G : 32;
        for (int off = Wg >> 1; off > 0; off >>= 1) {
            g += __shfl_xor_sync(FULL, g, off);
            bb += __shfl_xor_sync(FULL, bb, off);
        }
        if (G <= 32) {
            if (r == 0 && s < nage) {
                a.pDots[(size_t)bid * DOTS + 2 * s] = g;
                a.pDots[(size_t)bid * DOTS + 2 * s + 1] = bb;
            }
        } else {
            if (lane == 0) {
                s_red[2 * warp] = g;
                s_red[2 * warp + 1] = bb;
            }
            __syncthreads();
            const int wpa = G / 32;
            if (tid < 2 * nage) {
                const int s2 = tid >> 1, which = tid & 1;
                double acc = 0.0;
                for (int w = 0; w < wpa; ++w) acc += s_red[2 * (s2 * wpa + w) + which];
                a.pDots[(size_t)bid * DOTS + tid] = acc;
            }
        }
    }

    // ---- last block: Gram update, least squares, end of the iteration
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&st->ctr_fin, 1u) == (unsigned)nblk - 1u) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (ring) {
        // fixed-order two-level sum over the blocks: 8 interleaved sub-sums, then in order
        for (int t = tid; t < 2 * nage * 8; t += blockDim.x) {
            const int v = t >> 3, sp = t & 7;
            double acc = 0.0;
#pragma unroll 8
            for (int b = sp; b < nblk; b += 8) acc += __ldcg(a.pDots + (size_t)b * DOTS + v);
            s_part[t] = acc;
        }
        __syncthreads();
        for (int v = tid; v < 2 * nage; v += blockDim.x) {
            double acc = 0.0;
            for (int sp = 0; sp < 8; ++sp) acc += s_part[v * 8 + sp];
            s_red[v] = acc;
        }
        __syncthreads();
        if (tid == 0) {
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
        }
        __syncthreads();
        // theta: the certified Gram route (one warp), else Householder QR over the ring (whole block)
        const int mt = min(min(st->m, st->t), st->ring_count);
        if (warp == 0) {
            s_sl[lane] = (hnew - lane + m_max) % m_max;
            if (lane == 0) s_unc = 0;
            __syncwarp();
            int rank = 0;
            if (mt > 0 && a.ls_mode != LS_QR) {
                const double ct = a.ls_mode == LS_GRAM ? 0.0 : LS_CERT_TOL;
                rank = m_max <= 16 ? ls_warp_reg<16>(st, hnew, m_max, mt, a.rank_tol, ct, &s_unc, s_M, s_th)
                                   : ls_warp(st, hnew, m_max, mt, a.rank_tol, ct, &s_unc, s_M, s_inv, s_th);
            }
            if (mt == 0) s_th[lane] = 0.0;
            if (lane == 0) s_rank = rank;
        }
        __syncthreads();
        if (mt > 0 && (a.ls_mode == LS_QR || s_unc)) {
            const int rank = ls_qr_block(a.dF, s_sl, mt, a.Fprev, n, a.rank_tol, a.qrw, s_th);
            if (tid == 0) {
                s_rank = rank;
                st->ls_qr += 1;
            }
            __syncthreads();
        }
        if (warp == 0) {
            st->theta[lane] = s_th[lane];
            if (lane == 0) st->m_t = mt;
        }
    } else if (tid == 0) {
        s_rank = 0;
        st->m_t = 0;
    }
    __syncthreads();
    const int rank = s_rank;
    bool stop = false;
    if (init) {
        if (tid == 0) {
            st->t = 1;
            st->cur = 1;
            st->revert = 0;
        }
    } else {
        stop = st->t >= a.max_iter;
        __syncthreads();
        if (tid == 0) {
            st->ctr_fin = 0u;
            st->rank = rank;
            st->from_lloyd = rank == 0;
            st->E_prev2 = st->E_prev;
            st->E_prev = st->E_cur;
            if (stop) {
                st->done = 1;                // (P^t, G^t)
                st->converged = 0;
                st->final_src = 1;
                if (a.use_cond) cudaGraphSetConditional(a.cond, 0);
            } else {
                st->t += 1;
                st->cur ^= 1;
                st->revert = 0;
            }
        }
    }
    if (init && tid == 0) st->ctr_fin = 0u;
    // ---- small K*d: the accelerated iterate here, saving a launch.  Element-parallel (one
    // element per thread, FP64), then ||c'||^2 per centroid from the packed FP32 values.
    if (a.fuse_mix && !stop) {
        const int rk = init ? 0 : rank;
#pragma unroll 4
        for (size_t i = tid; i < n; i += blockDim.x) {
            const int j = (int)(i / d), k = (int)(i % d);
            const double g = __ldcg(a.CAU + i);
            double dg[MMAX];
#pragma unroll
            for (int q = 0; q < MMAX; ++q) dg[q] = q < rk ? __ldcg(a.dG + (size_t)s_sl[q] * n + i) : 0.0;
            double c = g;
#pragma unroll
            for (int q = 0; q < MMAX; ++q)
                if (q < rk) c -= s_th[q] * dg[q];
            a.C64[i] = c;
            if (a.fp32_path) {
                const double o = (double)a.origin[k];
                a.c32[0][i] = (float)c;
                a.c32[1][i] = (float)g;
                a.cpk[0][pk_index(j, k, a.DP)] = -2.f * (float)(c - o);
                a.cpk[1][pk_index(j, k, a.DP)] = -2.f * (float)(g - o);
            }
        }
        if (a.fp32_path) {
            __syncthreads();
            for (int j = tid; j < K; j += blockDim.x) {
                double n0 = 0.0, n1 = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double c0 = -0.5 * (double)a.cpk[0][pk_index(j, k, a.DP)];
                    const double c1 = -0.5 * (double)a.cpk[1][pk_index(j, k, a.DP)];
                    n0 += c0 * c0;
                    n1 += c1 * c1;
                }
                a.cpk[0][pk_index(j, d, a.DP)] = (float)n0;
                a.cpk[1][pk_index(j, d, a.DP)] = (float)n1;
            }
        }
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_fin(FinArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    fin_body(a, blockIdx.x, gridDim.x, smem);
}

// Persistent batched finalize over work items (instance, block of that instance).
__global__ void __launch_bounds__(FIN_THREADS) k_fin_batch(BatchFin b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const int2 w = b.items[it];
        FinArgs a = b.args[w.x];
        a.mode = b.mode;
        a.use_cond = 0;
        fin_body(a, w.y, a.nblk, smem);
        __syncthreads();
    }
}

// Block `bid` (256 threads, 8 centroids) of the mix.
__device__ __forceinline__ void mix_body(const MixArgs& a, const int bid)
{
    SolveState* st = a.st;
    if (st->done) return;
    __shared__ double s_th[MMAX];
    __shared__ int s_sl[MMAX];
    const int rank = a.mode == MODE_INIT ? 0 : st->rank;
    const int head = st->ring_head, m_max = a.m_max;
    if (threadIdx.x < MMAX) {
        s_th[threadIdx.x] = threadIdx.x < rank ? st->theta[threadIdx.x] : 0.0;
        s_sl[threadIdx.x] = (head - (int)threadIdx.x + m_max) % m_max;
    }
    __syncthreads();
    const int j = (bid * blockDim.x + threadIdx.x) >> 5;
    if (j < a.K)
        mix_pack_centroid(j, a.K, a.d, a.DP, a.fp32_path, a.C64, a.CAU, a.dG, s_th, s_sl, rank, a.origin, a.cpk,
                          a.c32);
}

__global__ void __launch_bounds__(256) k_mix(MixArgs a)
{
    mix_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_mix_batch(BatchMix b)
{
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const int2 w = b.items[it];
        MixArgs a = b.args[w.x];
        a.mode = b.mode;
        mix_body(a, w.y);
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void prep_body(const T* C0, int K, int d, int Kpad, int DP, int fp32_path, double* C64,
                                          float* origin, float* cpk0, float* cpk1, float* c32_0, SolveState* st,
                                          int m_init, int m_max)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double s_red[32];
    __shared__ float s_o[64];
    // zero the controller state
    unsigned int* sw = reinterpret_cast<unsigned int*>(st);
    for (size_t i = tid; i < sizeof(SolveState) / 4; i += blockDim.x) sw[i] = 0u;
    // origin o = mean of the initial centroids (FP64, fixed-order block reduction), rounded to FP32
    if (fp32_path) {
        for (int k = 0; k < d; ++k) {
            double v = 0.0;
            for (int j = tid; j < K; j += blockDim.x) v += (double)C0[(size_t)j * d + k];
            v = warp_sum(v);
            if (lane == 0) s_red[warp] = v;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
                s_o[k] = (float)(t / K);
                origin[k] = s_o[k];
            }
            __syncthreads();
        }
    }
    const size_t n = (size_t)K * d;
    for (size_t i = tid; i < n; i += blockDim.x) C64[i] = (double)C0[i];
    if (fp32_path) {
        for (size_t i = tid; i < (size_t)Kpad * DP; i += blockDim.x) {
            const int w = (int)(i % (2 * DP));
            const int j = (int)(i / (2 * DP)) * 2 + (w & 1), k = w >> 1;
            const float v = (j >= K && k == d) ? __int_as_float(0x7f800000) : 0.f;
            cpk0[i] = v;
            cpk1[i] = v;
        }
        __syncthreads();
        for (int j = tid; j < K; j += blockDim.x) {
            double nrm = 0.0;
            for (int k = 0; k < d; ++k) {
                const double c = (double)C0[(size_t)j * d + k];
                const float cc = (float)(c - (double)s_o[k]);
                c32_0[(size_t)j * d + k] = (float)c;
                cpk0[pk_index(j, k, DP)] = -2.f * cc;
                nrm += (double)cc * (double)cc;
            }
            cpk0[pk_index(j, d, DP)] = (float)nrm;
        }
    }
    __syncthreads();
    if (tid == 0) {
        st->m = m_init < m_max ? m_init : m_max;
        if (st->m < 0) st->m = 0;
        st->from_lloyd = 1;
        st->E_prev = st->E_prev2 = __longlong_as_double(0x7ff0000000000000LL);
        st->ring_head = m_max > 0 ? m_max - 1 : 0;      // first insert goes to slot 0
        st->status = KM_OK;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_prep(const T* C0, int K, int d, int Kpad, int DP, int fp32_path,
                                               double* C64, float* origin, float* cpk0, float* cpk1, float* c32_0,
                                               SolveState* st, int m_init, int m_max)
{
    prep_body<T>(C0, K, d, Kpad, DP, fp32_path, C64, origin, cpk0, cpk1, c32_0, st, m_init, m_max);
}

// One block per instance: the pass counter, then what k_prep does for a single solve.
__global__ void __launch_bounds__(1024) k_prep_batch(BatchPrep b)
{
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const PrepArgs p = b.args[b.items[it].x];
        if (threadIdx.x < 64) p.counter[threadIdx.x] = 0u;
        if (p.f64)
            prep_body<double>(reinterpret_cast<const double*>(p.C0), p.K, p.d, p.Kpad, p.DP, 0, p.C64, p.origin,
                              p.cpk0, p.cpk1, p.c32_0, p.st, p.m_init, p.m_max);
        else
            prep_body<float>(reinterpret_cast<const float*>(p.C0), p.K, p.d, p.Kpad, p.DP, p.pack, p.C64, p.origin,
                             p.cpk0, p.cpk1, p.c32_0, p.st, p.m_init, p.m_max);
        __syncthreads();
    }
}

struct DevInfo {
    int iters, accepted, rejected, passes, converged, m_final, status, ls_qr;
    double E;
    long long rescored;
    long long scanned;
};

template <typename T>
__device__ __forceinline__ void epi_body(const SolveState* st, const double* C64, const double* CAU, T* C_out,
                                         size_t n, const int32_t* rhoA, const int32_t* rhoB, int32_t* rho_out,
                                         int64_t N, DevInfo* info, int bid, int nblk)
{
    const double* src = st->final_src ? CAU : C64;
    const int32_t* rho = st->cur ? rhoB : rhoA;
    const size_t tid = (size_t)bid * blockDim.x + threadIdx.x, T_ = (size_t)nblk * blockDim.x;
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
        f.ls_qr = st->ls_qr;
        f.E = st->E_final;
        f.rescored = st->rescored;
        f.scanned = st->scanned;
        *info = f;
    }
}

template <typename T>
__global__ void k_epi(const SolveState* st, const double* C64, const double* CAU, T* C_out, size_t n,
                      const int32_t* rhoA, const int32_t* rhoB, int32_t* rho_out, int64_t N, DevInfo* info)
{
    epi_body<T>(st, C64, CAU, C_out, n, rhoA, rhoB, rho_out, N, info, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_epi_batch(BatchEpi b)
{
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const int2 w = b.items[it];
        const EpiArgs& e = b.args[w.x];
        if (e.f64)
            epi_body<double>(e.st, e.C64, e.CAU, reinterpret_cast<double*>(e.C_out), e.n, e.rhoA, e.rhoB, e.rho_out,
                             e.N, reinterpret_cast<DevInfo*>(e.info), w.y, e.nblk);
        else
            epi_body<float>(e.st, e.C64, e.CAU, reinterpret_cast<float*>(e.C_out), e.n, e.rhoA, e.rhoB, e.rho_out,
                            e.N, reinterpret_cast<DevInfo*>(e.info), w.y, e.nblk);
    }
}

// End of one batched loop pass: every instance done (or the guard) ends the while loop.
__global__ void __launch_bounds__(256) k_batch_done(BatchDone b)
{
    __shared__ int s_open;
    if (threadIdx.x == 0) s_open = 0;
    __syncthreads();
    const unsigned int loops = *b.loops + 1u;
    const bool guard = loops > b.max_loops;
    int open = 0;
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
        SolveState* st = b.st[i];
        if (!st) continue;
        if (!st->done) {
            if (guard) {
                st->status = KM_ETIMEOUT;
                st->done = 1;
            } else {
                open = 1;
            }
        }
    }
    if (open) atomicOr(&s_open, 1);
    __syncthreads();
    if (b.flags)
        for (int i = threadIdx.x; i < b.n; i += blockDim.x) b.flags[i] = b.st[i] ? b.st[i]->done : 0;
    if (threadIdx.x == 0) {
        *b.loops = loops;
        if (!s_open) {
            *b.all_done = 1;
            if (b.use_cond) cudaGraphSetConditional(b.cond, 0);
        }
    }
}

// kmeans_lsq: Eq. 7 for a caller's history by one block, with the solver's routines.  The Gram
// matrix and right-hand side are formed in full (p <= q dot products of length n), placed in the
// ring slots the solver's Cholesky reads (column c at slot (m - c) mod m, newest at slot 0), then
// the certified Gram route or the Householder QR as in k_fin.
__global__ void __launch_bounds__(FIN_THREADS) k_lsq(LsqArgs a)
{
    constexpr int CW = 8;
    __shared__ double s_red[(FIN_THREADS / 32) * CW];
    __shared__ double s_M[MMAX * MMAX];
    __shared__ double s_inv[MMAX];
    __shared__ double s_th[MMAX];
    __shared__ int s_sl[MMAX];
    __shared__ int s_unc, s_rank;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int m = a.m;
    const size_t n = a.n;
    SolveState* st = a.st;
    auto slot = [&](int c) { return (m - c) % m; };
    if (a.mode != LS_QR) {
        for (int p = 0; p < m; ++p) {
            const double* ap = a.dF + (size_t)p * n;
            for (int q0 = p; q0 <= m; q0 += CW) {          // q = m: the right-hand side <dF_p, f>
                double acc[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) acc[c] = 0.0;
                for (size_t i = tid; i < n; i += blockDim.x) {
                    const double v = ap[i];
#pragma unroll
                    for (int c = 0; c < CW; ++c) {
                        const int q = q0 + c;
                        if (q <= m) acc[c] = fma(v, q < m ? a.dF[(size_t)q * n + i] : a.f[i], acc[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    const double v = warp_sum(acc[c]);
                    if (lane == 0) s_red[warp * CW + c] = v;
                }
                __syncthreads();
                if (tid < CW && q0 + tid <= m) {
                    double v = 0.0;
                    for (int w = 0; w < nw; ++w) v += s_red[w * CW + tid];
                    const int q = q0 + tid;
                    if (q == m) {
                        st->bvec[slot(p)] = v;
                    } else {
                        st->gram[slot(p) * MMAX + slot(q)] = v;
                        st->gram[slot(q) * MMAX + slot(p)] = v;
                    }
                }
                __syncthreads();
            }
        }
    }
    if (warp == 0) {
        s_sl[lane] = lane;                                   // the caller's column q is at dF + q n
        if (lane == 0) s_unc = 0;
        __syncwarp();
        int rank = 0;
        if (a.mode != LS_QR) {
            const double ct = a.mode == LS_GRAM ? 0.0 : LS_CERT_TOL;
            rank = m <= 16 ? ls_warp_reg<16>(st, 0, m, m, a.rank_tol, ct, &s_unc, s_M, s_th)
                           : ls_warp(st, 0, m, m, a.rank_tol, ct, &s_unc, s_M, s_inv, s_th);
        }
        if (lane == 0) s_rank = rank;
    }
    __syncthreads();
    const int qr = a.mode == LS_QR || s_unc;
    if (qr) {
        const int rank = ls_qr_block(a.dF, s_sl, m, a.f, n, a.rank_tol, a.W, s_th);
        if (tid == 0) s_rank = rank;
        __syncthreads();
    }
    if (tid < m) a.theta[tid] = s_th[tid];
    if (tid == 0) {
        if (a.rank) *a.rank = s_rank;
        if (a.qr_used) *a.qr_used = qr;
    }
}

}  // namespace

int fin_blocks(int K, int d, int* KB)
{
    int kb = d > 16 ? 8 : 16 / (d + 1);
    if (kb < 1) kb = 1;
    *KB = kb;
    return (K + kb - 1) / kb;
}

size_t fin_smem(int KB, int d)
{
    const int E = KB * (d + 1);
    return sizeof(double) * ((size_t)E + 2 * (size_t)KB * d + 2 * FIN_THREADS + 2 * MMAX * 8);
}

// A launch whose dynamic shared memory plus the kernel's static shared memory exceeds 48 KB needs
// the kernel's opt-in limit raised first.
cudaError_t allow_dyn_smem(const void* fn, size_t dyn)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes + dyn <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t launch_fin(const FinArgs& a, int nblocks, cudaStream_t s)
{
    const size_t smem = fin_smem(a.KB, a.d);
    cudaError_t e = allow_dyn_smem(reinterpret_cast<const void*>(k_fin), smem);
    if (e != cudaSuccess) return e;
    k_fin<<<nblocks, FIN_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mix(const MixArgs& a, cudaStream_t s)
{
    const int blocks = (a.K * 32 + 255) / 256;
    k_mix<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prep(const void* C0, bool f64, int K, int d, int Kpad, int DP, double* C64,
                        float* origin, float* cpk0, float* cpk1, float* c32_0, SolveState* st, int m_init,
                        int m_max, cudaStream_t s, int pack)
{
    if (f64)
        k_prep<double><<<1, 1024, 0, s>>>(reinterpret_cast<const double*>(C0), K, d, Kpad, DP, 0, C64, origin,
                                          cpk0, cpk1, c32_0, st, m_init, m_max);
    else
        k_prep<float><<<1, 1024, 0, s>>>(reinterpret_cast<const float*>(C0), K, d, Kpad, DP, pack, C64, origin,
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

cudaError_t launch_lsq(const LsqArgs& a, cudaStream_t s)
{
    k_lsq<<<1, FIN_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fin_batch(const BatchFin& b, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = allow_dyn_smem(reinterpret_cast<const void*>(k_fin_batch), smem);
    if (e != cudaSuccess) return e;
    k_fin_batch<<<grid, FIN_THREADS, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_mix_batch(const BatchMix& b, int grid, cudaStream_t s)
{
    k_mix_batch<<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_prep_batch(const BatchPrep& b, cudaStream_t s)
{
    const int grid = b.nitems < 1024 ? b.nitems : 1024;
    k_prep_batch<<<grid, 1024, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_epi_batch(const BatchEpi& b, int grid, cudaStream_t s)
{
    k_epi_batch<<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch_done(const BatchDone& b, cudaStream_t s)
{
    k_batch_done<<<1, 256, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace km
