// Host runtime shared by the solver entry points (api.cu) and the batched / serving entry points
// (batch.cu): context, workspace plans, arena addressing, launch argument resolution and the
// launch sequences of one solve (prologue, loop body, epilogue).
#pragma once

#include "dense.cuh"
#include "km_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace km;

namespace {

struct GraphKey {
    const void* X;
    const void* Xb;
    const void* Xl;
    int64_t N;
    int d, K, prec;
    const void* C0;
    void* C_out;
    int32_t* rho_out;
    kmeans_params p;
    void* arena;
    size_t arena_bytes;
    int ham;
    int lsq;
};

struct Plan {
    // offsets into the arena
    size_t st, rhoA, rhoB, C64, CAU, Fprev, dF, dG, cpk0, cpk1, c32_0, c32_1, origin;
    size_t pS, pCnt, pE, pNch, pResc, pScan, pBad, pDots, counter, info, acc, qrw;
    size_t hX, hXb, hC0, hCout, hRho;   // device copies for kmeans_solve_host
    // dense path (tensor-core assignment, sort-based update)
    size_t cb0, cb1, cl0, cl1, xlo, cn0, cn1, queue, rkey, qcount, err, hist, counts, off, choff, chunk_cluster, nchunks, perm,
        part, pe, pnch, rowe, rown, xn2, drift, map, nrows, xch, xcl;
    size_t spair0, spair1, npair0, npair1, dsum, dcnt, qx;   // incremental update of the solver passes
    size_t total;
    int nb, nfin, KB, Kpad, DP;
    bool dense;
    int dpad, nbk, rpb, max_chunks;
    size_t smem;
    // Hamerly bounds of the FP32 solver passes (hg > 0: group bounds in place of the single lower bound)
    bool ham;
    int hq_cap;
    int hg;
    size_t hub, hlb, hlast, hprep, hlbg, hgd, hperm, hgoff;
};

constexpr int DENSE_RPB = 1024;   // rows per block of the dense update's histogram and scatter (at least K)
constexpr int QX_BLOCKS = 4096;   // room for k_xcheck's block partials of sum ||x||^2
constexpr int DENSE_SEG = 64;     // rows per segment-sum chunk

}  // namespace

struct kmeans_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    size_t budget = 0;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    int nsm = 0;
    std::string err;
    bool have_graph = false;
    GraphKey key{};
    cudaGraphExec_t exec = nullptr;
    void* h_info = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::mutex mu;
    // batched solves: the graph of the last batch shape and its launch shapes
    bool have_bgraph = false;
    std::string bkey;
    cudaGraphExec_t bexec = nullptr;
    std::string bdesc;
    std::vector<int> bgrids;
    void* h_binfo = nullptr;
    size_t h_binfo_bytes = 0;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

kmeans_status fail(kmeans_ctx* c, kmeans_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

kmeans_status cuda_fail(kmeans_ctx* c, cudaError_t e, const char* where)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    return fail(c, KM_ECUDA, buf);
}

#define KM_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

kmeans_status check_data(kmeans_ctx* ctx, const kmeans_data* X, int K, bool need_bf16)
{
    if (!X || !X->X) return fail(ctx, KM_EINVAL, "X is NULL");
    if (X->N < 1 || X->d < 1 || X->d > 4096) return fail(ctx, KM_EINVAL, "need N >= 1 and 1 <= d <= 4096");
    if (K < 1 || (int64_t)K > X->N) return fail(ctx, KM_EINVAL, "need 1 <= K <= N");
    if (X->prec != KM_F64 && X->prec != KM_F32 && X->prec != KM_BF16_F32)
        return fail(ctx, KM_EINVAL, "unknown precision");
    if (X->prec == KM_BF16_F32 && need_bf16 && !X->X_bf16) return fail(ctx, KM_EINVAL, "X_bf16 is NULL");
    if (X->prec == KM_BF16_F32 && X->d > 16 &&
        (((uintptr_t)X->X | (uintptr_t)X->X_bf16 | (uintptr_t)X->X_bf16_lo) & 15u))
        return fail(ctx, KM_EINVAL, "the tensor-core path needs X, X_bf16 and X_bf16_lo 16-byte aligned");
    return KM_OK;
}

// Blocks of a low-d pass: as many as are resident at once (the kernel's occupancy for this shared
// memory size, at most 4 per SM), and at least 1024 rows per block on the FP32 path (256 on the
// FP64 path) so that the per-block staging and partial sums stay small against the scan.  The
// count fixes the order of the update's sums; batched solves reuse it per instance.
int pass_blocks(kmeans_ctx* ctx, int64_t N, size_t smem, int prec, int d, bool ao = false)
{
    int per_sm = ao ? pass_lowd_occupancy_ao(d, smem) : pass_lowd_occupancy(prec, d, smem);
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    int64_t nb = (int64_t)ctx->nsm * per_sm;
    const int64_t rows = prec == KM_F64 ? LOWD_THREADS : 4 * LOWD_THREADS;
    const int64_t need = (N + rows - 1) / rows;
    if (nb > need) nb = need;
    if (nb < 1) nb = 1;
    return (int)nb;
}

// Workspace layout of one problem shape (bins = fused per-block update partials).
// Dense path: BF16 tensor-core assignment, sort-based update (d in 17..128, d % 8 == 0).
kmeans_status make_plan_dense(kmeans_ctx* ctx, int64_t N, int d, int K, int m_max, bool host_copies, Plan& P)
{
    if (d > 128 || d % 8 != 0)
        return fail(ctx, KM_EINVAL, "the tensor-core path needs d <= 128 and d % 8 == 0");
    if (K > 4096) return fail(ctx, KM_EINVAL, "the tensor-core path supports K <= 4096");
    P.dense = true;
    P.dpad = (d + 63) / 64 * 64;
    P.Kpad = (K + 255) / 256 * 256;
    P.DP = 0;
    P.nb = 1;
    P.nfin = fin_blocks(K, d, &P.KB);
    // the per-block histograms hold K * nbk counts: rows per block >= K keeps them within N entries
    P.rpb = std::max(DENSE_RPB, (K + 255) / 256 * 256);
    P.nbk = (int)((N + P.rpb - 1) / P.rpb);
    P.max_chunks = (int)((N + DENSE_SEG - 1) / DENSE_SEG) + K;
    P.smem = 0;
    const size_t n = (size_t)K * d;
    const int mm = m_max > 0 ? m_max : 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    P.counter = take(256);
    P.st = take(sizeof(SolveState));
    P.rhoA = take((size_t)N * 4);
    P.rhoB = take((size_t)N * 4);
    P.C64 = take(n * 8);
    P.CAU = take(n * 8);
    P.Fprev = take(n * 8);
    P.dF = take((size_t)mm * n * 8);
    P.dG = take((size_t)mm * n * 8);
    P.qrw = take((size_t)(mm + 1) * n * 8);
    P.cpk0 = P.cpk1 = 0;
    P.c32_0 = take(n * 4);
    P.c32_1 = take(n * 4);
    P.origin = take(256);
    P.cb0 = take((size_t)P.Kpad * P.dpad * 2);
    P.cb1 = take((size_t)P.Kpad * P.dpad * 2);
    P.cl0 = take((size_t)P.Kpad * P.dpad * 2);
    P.cl1 = take((size_t)P.Kpad * P.dpad * 2);
    P.xlo = take((size_t)N * d * 2);     // x_lo = bf16(x - x_hi), when the caller does not supply it
    P.cn0 = take((size_t)P.Kpad * 4);
    P.cn1 = take((size_t)P.Kpad * 4);
    P.queue = take((size_t)N * 4);       // near-tie rows
    P.rkey = take((size_t)N * 8);        // their (distance, index) keys
    P.qcount = take(256);
    P.err = take(256);
    P.hist = take((size_t)K * P.nbk * 4);
    P.counts = take((size_t)K * 4);
    P.off = take((size_t)(K + 1) * 4);
    P.choff = take((size_t)K * 4);
    P.chunk_cluster = take((size_t)P.max_chunks * 4);
    P.nchunks = take(256);
    P.perm = take((size_t)N * 4);
    P.part = take((size_t)P.max_chunks * d * 4);
    P.pe = take((size_t)P.max_chunks * 8);
    P.pnch = take((size_t)P.nbk * 8);
    P.acc = take(n * 8 + (size_t)K * 4);     // fixed-point residual sums + counts of a pass
    // Hamerly bounds of the solver passes: per-row bounds and norms, the last pass's centroids and
    // their drifts, the rows to scan and their BF16 parts in compact buffers
    P.hub = take((size_t)N * 4);
    P.hlb = take((size_t)N * 4);
    P.xn2 = take((size_t)N * 4);
    P.hlast = take(n * 4);
    P.drift = take((size_t)K * 4);
    P.map = take((size_t)N * 4);
    P.nrows = take(256);
    P.xch = take((size_t)N * d * 2);
    P.xcl = take((size_t)N * d * 2);
    P.rowe = take(4096 * 8);
    P.rown = take(4096 * 8);
    // incremental update: the integer sums and sizes of the partitions in rhoA / rhoB, a pass's
    // change of them, and sum ||x||^2 with k_xcheck's block partials
    P.spair0 = take(n * 8);
    P.spair1 = take(n * 8);
    P.npair0 = take((size_t)K * 4);
    P.npair1 = take((size_t)K * 4);
    P.dsum = take(n * 8);
    P.dcnt = take((size_t)K * 4);
    P.qx = take((size_t)(1 + QX_BLOCKS) * 8);
    P.pS = 0;
    P.pCnt = P.counts;
    P.pE = P.pNch = P.pResc = P.pScan = P.pBad = 0;
    P.pDots = take((size_t)P.nfin * DOTS * 8);
    P.info = take(256);
    if (host_copies) {
        P.hX = take((size_t)N * d * 4);
        P.hXb = take((size_t)N * d * 2);
        P.hC0 = take(n * 4);
        P.hCout = take(n * 4);
        P.hRho = take((size_t)N * 4);
    } else {
        P.hX = P.hXb = P.hC0 = P.hCout = P.hRho = 0;
    }
    P.total = o;
    return KM_OK;
}

// KM_LSQ in the environment picks the least-squares route of Eq. 7: "qr" = Householder QR always,
// "gram" = the Cholesky factor of the Gram matrix always; unset = the Gram route when it certifies
// its factor, else QR (the results agree to about 1e-10 relative on well-conditioned histories).
int ls_mode()
{
    const char* v = getenv("KM_LSQ");
    if (v && !strcmp(v, "qr")) return LS_QR;
    if (v && !strcmp(v, "gram")) return LS_GRAM;
    return LS_AUTO;
}

// KM_HAMERLY=0 in the environment solves without Hamerly bounds (same results, every row scanned).
bool hamerly_mode()
{
    const char* v = getenv("KM_HAMERLY");
    return !(v && v[0] == '0');
}

// KM_DINC in the environment picks the update of the dense solver passes: 0 = the sorted update
// over every row (the residual sums); unset or 1 = the incremental update, which rebuilds its sums
// in full when more than a tenth of the rows changed; 2 = the incremental update rebuilding in full
// every pass; 3 = incremental after the first pass whatever the changes.  1, 2 and 3 give the same
// integer sums, hence bitwise the same solves.
int dense_inc_mode()
{
    const char* v = getenv("KM_DINC");
    if (!v || !v[0]) return 1;
    return (v[0] >= '0' && v[0] <= '3') ? v[0] - '0' : 1;
}

// KM_BOUNDS in the environment picks the bounds of standalone FP32 solves: "group" = group bounds at
// any K, "hamerly" = Hamerly's bounds at any K (half distances however costly); unset = the rule below.
int bounds_env()
{
    const char* v = getenv("KM_BOUNDS");
    if (v && !strcmp(v, "group")) return 2;
    if (v && !strcmp(v, "hamerly")) return 1;
    return 0;
}

// Solver plans (ham_ok) on the FP32 low-d path use Hamerly bounds when the centroids' pairwise
// half-distances stay affordable (K*K*d <= 2^23: the TRIAL pass's last block recomputes them alone
// when a REVERT pass follows) and the pass fits in shared memory.  Above that, plans that allow it
// (group_ok: the standalone solver, whose prologue forms the groups) use group bounds: one lower
// bound per group of nearby centroids (hg = K/64 groups, 2..16), no half distances.  (The low-d
// pass's own shared memory caps K near 1,100 at d = 3, so group bounds are mostly reached through
// KM_BOUNDS=group; measured on GB300 they cost more per pass than the single Hamerly bound.)
kmeans_status make_plan(kmeans_ctx* ctx, int64_t N, int d, int K, int prec, int m_max, bool host_copies,
                        Plan& P, bool bins = true, bool ham_ok = false, bool group_ok = false)
{
    P.dense = false;
    P.ham = false;
    P.hq_cap = 0;
    P.hg = 0;
    P.hub = P.hlb = P.hlast = P.hprep = P.hlbg = P.hgd = P.hperm = P.hgoff = 0;
    P.dpad = P.nbk = P.rpb = P.max_chunks = 0;
    if (prec == KM_BF16_F32 && d > 16) return make_plan_dense(ctx, N, d, K, m_max, host_copies, P);
    if (d > 16) return fail(ctx, KM_EINVAL, "d > 16 needs KM_BF16_F32 (the tensor-core path)");
    const bool f32 = prec != KM_F64;
    const size_t esz = f32 ? 4 : 8;
    P.DP = pass_lowd_dp(d);
    P.Kpad = (K + KPAD_ALIGN - 1) / KPAD_ALIGN * KPAD_ALIGN;
    P.smem = pass_lowd_smem(prec, d, K, P.Kpad, bins);
    if (P.smem > (size_t)LOWD_SMEM_MAX)
        return fail(ctx, KM_EINVAL, bins ? "K*d too large for the fused low-d update" : "K*d too large");
    // FP32 plans without update bins (the standalone assignment and energy calls) run the
    // assignment-only kernel, with its own resident blocks per SM
    P.nb = pass_blocks(ctx, N, P.smem, prec, d, f32 && !bins);
    const int benv = group_ok ? bounds_env() : 0;
    const bool cheap_half = (int64_t)K * K * d <= (int64_t(1) << 23) || benv == 1;
    const bool group = group_ok && K >= 2 && K <= 16384 && benv != 1 && (!cheap_half || benv == 2);
    if (ham_ok && f32 && bins && hamerly_mode() && (cheap_half || group) && N < (int64_t(1) << 31)) {
        const int64_t per = (int64_t)P.nb * LOWD_THREADS;
        const int hg = group ? std::min(std::max(K / 64, 2), std::min(16, K)) : 0;
        // rows a block queues for full scans per round (the passes drain the queue in rounds): all of
        // a block's rows when they fit in shared memory, else as many whole rows per thread as fit
        // (group bounds: at most 2048); Hamerly's rounds take hq_cap / LOWD_THREADS rows per thread
        int cap = (int)((N + per - 1) / per) * LOWD_THREADS;
        if (hg > 0) cap = std::min(cap, 2048);
        if (const char* v = getenv("KM_HQ_CAP"))            // smaller rounds (tests)
            cap = std::max(LOWD_THREADS, std::min(cap, atoi(v) / LOWD_THREADS * LOWD_THREADS));
        // the queue may not lower the blocks per SM the grid was sized for
        const int per_sm = std::max(1, (int)std::min<int64_t>(4, (P.nb + ctx->nsm - 1) / ctx->nsm));
        const size_t budget = std::min<size_t>(LOWD_SMEM_MAX, (SM_SMEM - 1024) / per_sm - 1024);
        const size_t sm1 = pass_lowd_smem(prec, d, K, P.Kpad, bins, LOWD_THREADS, hg);   // one row per thread
        if (sm1 <= budget) {
            const int fit = LOWD_THREADS + (int)((budget - sm1) / 4) / LOWD_THREADS * LOWD_THREADS;
            cap = std::min(cap, fit);
        }
        const size_t sm = pass_lowd_smem(prec, d, K, P.Kpad, bins, cap, hg);
        if (sm <= (size_t)LOWD_SMEM_MAX) {
            P.ham = true;
            P.hq_cap = cap;
            P.hg = hg;
            P.smem = sm;
        }
    }
    P.nfin = fin_blocks(K, d, &P.KB);
    const size_t n = (size_t)K * d;
    const int mm = m_max > 0 ? m_max : 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    P.counter = take(256);          // fixed offset 0 for every plan; zeroed at the start of every call
    if (P.ham) {
        P.hub = take((size_t)N * 4);
        P.hlb = take((size_t)N * 4);
        P.hlast = take(n * 4);
        P.hprep = take(((size_t)2 * P.Kpad + 8) * 4);
        if (P.hg > 0) {
            P.hlbg = take((size_t)N * P.hg * 4);
            P.hgd = take((size_t)P.hg * 4);
            P.hperm = take((size_t)K * 4);
            P.hgoff = take((size_t)(P.hg + 1) * 4);
        }
    }
    P.st = take(sizeof(SolveState));
    P.rhoA = take((size_t)N * 4);
    P.rhoB = take((size_t)N * 4);
    P.C64 = take(n * 8);
    P.CAU = take(n * 8);
    P.Fprev = take(n * 8);
    P.dF = take((size_t)mm * n * 8);
    P.dG = take((size_t)mm * n * 8);
    P.qrw = take((size_t)(mm + 1) * n * 8);
    P.cpk0 = take((size_t)P.Kpad * P.DP * 4);
    P.cpk1 = take((size_t)P.Kpad * P.DP * 4);
    P.c32_0 = take(n * 4);
    P.c32_1 = take(n * 4);
    P.origin = take(64 * 4);
    P.pS = take((size_t)P.nb * n * 8);       // FP64 bins, or FP32 bins / 64-bit fixed point (FP32 path)
    P.pCnt = take((size_t)P.nb * K * 4);
    P.pE = take((size_t)P.nb * 8);
    P.pNch = take((size_t)P.nb * 8);
    P.pResc = take((size_t)P.nb * 8);
    P.pScan = take((size_t)P.nb * 8);
    P.pBad = take((size_t)P.nb * 4);
    P.acc = (f32 && d <= FX_MAX_D) ? take(n * 8 + (size_t)K * 4) : 0;   // fixed-point totals + counts
    P.pDots = take((size_t)P.nfin * DOTS * 8);
    P.info = take(256);
    if (host_copies) {
        P.hX = take((size_t)N * d * esz);
        P.hXb = 0;
        P.hC0 = take(n * esz);
        P.hCout = take(n * esz);
        P.hRho = take((size_t)N * 4);
    } else {
        P.hX = P.hXb = P.hC0 = P.hCout = P.hRho = 0;
    }
    P.total = o;
    return KM_OK;
}

kmeans_status ensure_arena(kmeans_ctx* ctx, size_t bytes)
{
    if (ctx->arena && ctx->arena_bytes >= bytes) return KM_OK;
    if (ctx->budget && bytes > ctx->budget) {
        char buf[160];
        snprintf(buf, sizeof(buf), "workspace of %zu bytes exceeds the HBM budget of %zu bytes", bytes, ctx->budget);
        return fail(ctx, KM_ENOMEM, buf);
    }
    if (ctx->have_graph) {
        cudaGraphExecDestroy(ctx->exec);
        ctx->have_graph = false;
    }
    if (ctx->have_bgraph) {
        cudaGraphExecDestroy(ctx->bexec);
        ctx->have_bgraph = false;
        ctx->bkey.clear();
    }
    if (ctx->arena) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    e = cudaMemset(p, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemset");
    ctx->arena = p;
    ctx->arena_bytes = bytes;
    return KM_OK;
}

template <typename T>
T* at(char* base, size_t off)
{
    return reinterpret_cast<T*>(base + off);
}

inline char* arena_base(kmeans_ctx* ctx) { return static_cast<char*>(ctx->arena); }

PassArgs base_pass(char* base, const Plan& P, const void* X, int64_t N, int K, int prec)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.X = X;
    a.N = N;
    a.K = K;
    a.Kpad = P.Kpad;
    a.cpk[0] = at<float>(base, P.cpk0);
    a.cpk[1] = at<float>(base, P.cpk1);
    a.c32[0] = at<float>(base, P.c32_0);
    a.c32[1] = at<float>(base, P.c32_1);
    a.c64[0] = at<double>(base, P.C64);
    a.c64[1] = at<double>(base, P.CAU);
    a.origin = at<float>(base, P.origin);
    a.rho[0] = at<int32_t>(base, P.rhoA);
    a.rho[1] = at<int32_t>(base, P.rhoB);
    a.pS = at<void>(base, P.pS);
    a.pCnt = at<int32_t>(base, P.pCnt);
    a.pE = at<double>(base, P.pE);
    a.pNch = at<long long>(base, P.pNch);
    a.pResc = at<long long>(base, P.pResc);
    a.pScan = P.pScan ? at<long long>(base, P.pScan) : nullptr;
    a.pBad = at<int>(base, P.pBad);
    a.counter = at<unsigned int>(base, P.counter);
    a.st = at<SolveState>(base, P.st);
    (void)prec;
    return a;
}

// First-order rounding-error bound of the FP32 score ||c'||^2 - 2 x'.c' (u = 2^-24), with a 1%
// allowance for second-order terms:  D FMAs on partial sums <= ||c'||^2 + 2|x'||c'|, the rounding of
// ||c'||^2, of c' = fl(c - o) and of x' = fl(x - o):
//   |err| <= u * ((D + 3) max|c'|^2 + (2D + 4) |x'| max|c'|).
void set_bound(PassArgs& a, int d)
{
    const double u = 5.9604644775390625e-8;
    a.bound_coef = (float)(1.01 * (d + 3) * u);
    a.bound_coef2 = (float)(1.01 * (2 * d + 4) * u);
}


// Shared-memory class of a low-d pass (resident blocks per SM its smem allows, at most 4): the
// batched and serving launches group instances by (precision, d, class) so that a small instance is
// not launched with a large instance's shared memory.
inline int smem_class(size_t smem)
{
    const int c = (int)((SM_SMEM - 1024) / (smem + 1024));
    return c < 1 ? 1 : (c > 4 ? 4 : c);
}

// The accelerated iterate could be formed inside k_fin's last block (saving a launch), but FP64 is
// slow on this part (a few FP64 lanes per SM per cycle), so one block's mix over all K*d elements
// costs more than a launch of k_mix, which spreads it over K/8 blocks: only tiny problems fuse.
inline bool fuse_mix_rule(int K, int d) { return (size_t)K * d <= 64; }

// Everything one solve launches, resolved to device pointers once.
struct Launch {
    PassArgs pa;
    FinArgs fa;
    MixArgs ma;
    Plan P;
    kmeans_params p;
    const void* C0;
    void* C_out;
    int32_t* rho_out;
    SolveState* st;
    void* info;
    int32_t* rhoA;
    int32_t* rhoB;
    int64_t N;
    int d, K, prec, m_max;
    bool f64;
    // dense path
    DenseArgs da;
    PackArgs pk;
    const float* X32;
    int nsm;
    DenseMaps maps;
    DenseMaps maps_c;            // the same over the compact buffers of the rows a bounded pass scans
    bool dbounds = false;        // Hamerly bounds on the dense solver passes
    int* dmap = nullptr;         // their list of rows to scan, its length and the compact BF16 buffers
    unsigned int* dnrows = nullptr;
    void* dxch = nullptr;
    void* dxcl = nullptr;
    const void* xlo = nullptr;   // the low BF16 part of X the passes read
    bool xsplit = false;         // the prologue computes it into the workspace
    bool maps_ok = true;
};

// Dense-path arguments over the plan's buffers (centroid sets 0 = C^t, 1 = C_AU).
DenseArgs dense_args(char* base, const Plan& P, const float* X32, int64_t N, int d, int K)
{
    DenseArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N;
    a.d = d;
    a.dpad = P.dpad;
    a.K = K;
    a.Kpad = P.Kpad;
    a.X = X32;
    a.cn[0] = at<float>(base, P.cn0);
    a.cn[1] = at<float>(base, P.cn1);
    a.c32[0] = at<float>(base, P.c32_0);
    a.c32[1] = at<float>(base, P.c32_1);
    a.c64[0] = at<double>(base, P.C64);
    a.c64[1] = at<double>(base, P.CAU);
    // Rigorous bound on |s - s*| for the score s = fl(||c||^2 - 2 v), v the MMA's sum
    // x_hi.c_hi + x_lo.c_hi + x_hi.c_lo, s* = ||c||^2 - 2 x.c with x, c the FP32 values the rescoring
    // uses.  BF16 rounding to nearest has unit roundoff u_b = 2^-8: |x - x_hi| <= u_b |x|,
    // |x - x_hi - x_lo| <= u_b^2 |x| componentwise, likewise c.  Then
    //   |x.c - (x_hi.c_hi + x_lo.c_hi + x_hi.c_lo)| <= (3 u_b^2 + u_b^3) |x||c|       (dropped terms)
    //   FP32 accumulation of the 3d exact BF16 products inside the MMA, allowing 2u per addition
    //   (adders that truncate):                      <= 6 d u (1 + 4 u_b) |x||c|
    //   the epilogue's fma and the rounding of ||c||^2 (FP64 sum rounded once):
    //                                                 <= u (||c||^2 + 2 |x||c| (1 + alpha)) + u ||c||^2
    // so B = (2 alpha + 2 u (1 + alpha)) |x||c| + (2u + u^2) ||c||^2, alpha the first two lines.  The
    // epilogue takes |x| from the BF16 row (|x| <= |x_hi| / (1 - u_b), and the FP32 sum of squares
    // of d terms is within (1 + d u)) and max|c| over the centroids.
    const double ub = 1.0 / 256.0, u = 5.9604644775390625e-8;
    const double alpha = 3.0 * ub * ub + ub * ub * ub + 6.0 * d * u * (1.0 + 4.0 * ub);
    a.bcoef_a = (float)((2.0 * alpha + 2.0 * u * (1.0 + alpha)) / (1.0 - ub) * (1.0 + d * u) * 1.01);
    a.bcoef_b = (float)((2.0 * u + u * u) * 1.01);
    a.rho_pair[0] = at<int32_t>(base, P.rhoA);
    a.rho_pair[1] = at<int32_t>(base, P.rhoB);
    a.queue = at<int>(base, P.queue);
    a.rkey = at<void>(base, P.rkey);
    a.qcount = at<unsigned int>(base, P.qcount);
    a.err = at<int>(base, P.err);
    a.rows_per_block = P.rpb;
    a.hist = at<int>(base, P.hist);
    a.counts = at<int32_t>(base, P.counts);
    a.off = at<int>(base, P.off);
    a.choff = at<int>(base, P.choff);
    a.chunk_cluster = at<int>(base, P.chunk_cluster);
    a.nchunks = at<int>(base, P.nchunks);
    a.perm = at<int>(base, P.perm);
    a.part = at<float>(base, P.part);
    a.pe = at<double>(base, P.pe);
    a.pnch = at<long long>(base, P.pnch);
    a.acc = at<long long>(base, P.acc);
    a.accC = reinterpret_cast<int32_t*>(a.acc + (size_t)K * d);
    a.counter = at<unsigned int>(base, P.counter);
    a.st = at<SolveState>(base, P.st);
    a.inc = 0;                                  // set for the solver passes by make_launch
    a.inc_cap = N / 10;
    a.Spair[0] = at<long long>(base, P.spair0);
    a.Spair[1] = at<long long>(base, P.spair1);
    a.Npair[0] = at<int32_t>(base, P.npair0);
    a.Npair[1] = at<int32_t>(base, P.npair1);
    a.dS = at<long long>(base, P.dsum);
    a.dN = at<int32_t>(base, P.dcnt);
    a.qx = at<double>(base, P.qx);
    return a;
}

PackArgs pack_args(char* base, const Plan& P, int d, int K)
{
    PackArgs p;
    memset(&p, 0, sizeof(p));
    p.K = K;
    p.Kpad = P.Kpad;
    p.d = d;
    p.dpad = P.dpad;
    p.nsets = 2;
    p.src64[0] = at<double>(base, P.C64);
    p.src64[1] = at<double>(base, P.CAU);
    p.cb[0] = at<__nv_bfloat16>(base, P.cb0);
    p.cb[1] = at<__nv_bfloat16>(base, P.cb1);
    p.cl[0] = at<__nv_bfloat16>(base, P.cl0);
    p.cl[1] = at<__nv_bfloat16>(base, P.cl1);
    p.cn[0] = at<float>(base, P.cn0);
    p.cn[1] = at<float>(base, P.cn1);
    p.c32[0] = at<float>(base, P.c32_0);
    p.c32[1] = at<float>(base, P.c32_1);
    p.st = at<SolveState>(base, P.st);
    return p;
}

// The low BF16 part of X the dense pass reads: the caller's, or the workspace copy (then computed by
// launch_xsplit before the first pass).
const void* dense_xlo(char* base, const Plan& P, const kmeans_data* X)
{
    return X->X_bf16_lo ? X->X_bf16_lo : static_cast<const void*>(at<void>(base, P.xlo));
}

bool dense_maps(char* base, const Plan& P, const void* Xb, const void* Xl, int64_t N, int d, DenseMaps* m)
{
    return make_tmap_bf16(&m->xh, Xb, N, d, 128) && make_tmap_bf16(&m->xl, Xl, N, d, 128) &&
           make_tmap_bf16(&m->ch[0], at<void>(base, P.cb0), P.Kpad, P.dpad, 256) &&
           make_tmap_bf16(&m->ch[1], at<void>(base, P.cb1), P.Kpad, P.dpad, 256) &&
           make_tmap_bf16(&m->cl[0], at<void>(base, P.cl0), P.Kpad, P.dpad, 256) &&
           make_tmap_bf16(&m->cl[1], at<void>(base, P.cl1), P.Kpad, P.dpad, 256);
}

Launch make_launch(char* base, int nsm, const Plan& P, const kmeans_data* X, int K, const void* C0,
                   const kmeans_params& p, void* C_out, int32_t* rho_out)
{
    Launch L;
    L.P = P;
    L.p = p;
    L.C0 = C0;
    L.C_out = C_out;
    L.rho_out = rho_out;
    L.N = X->N;
    L.d = X->d;
    L.K = K;
    L.prec = X->prec;
    L.f64 = X->prec == KM_F64;
    L.m_max = p.lloyd_only ? 0 : p.m_max;
    L.st = at<SolveState>(base, P.st);
    L.info = at<void>(base, P.info);
    L.rhoA = at<int32_t>(base, P.rhoA);
    L.rhoB = at<int32_t>(base, P.rhoB);
    const int d = X->d;
    const int64_t thr = p.tol > 0 ? (int64_t)(p.tol * (double)X->N) : 0;

    PassArgs& pa = L.pa;
    pa = base_pass(base, P, X->X, X->N, K, X->prec);
    set_bound(pa, d);
    pa.m_max = L.m_max;
    pa.max_iter = p.max_iter;
    pa.lloyd_only = p.lloyd_only;
    pa.fixed_m = p.fixed_m ? 1 : 0;
    pa.eps1 = p.eps1;
    pa.eps2 = p.eps2;
    pa.thr = thr;
    pa.ham = P.ham ? 1 : 0;
    pa.hq_cap = P.hq_cap;
    pa.d = d;
    pa.hub = P.ham ? at<float>(base, P.hub) : nullptr;
    pa.hlb = P.ham ? at<float>(base, P.hlb) : nullptr;
    pa.hlast = P.ham ? at<float>(base, P.hlast) : nullptr;
    pa.hdr = P.ham ? at<float>(base, P.hprep) : nullptr;
    pa.hs = P.ham ? pa.hdr + P.Kpad : nullptr;
    pa.hm = P.ham ? pa.hdr + 2 * P.Kpad : nullptr;
    pa.hg = P.hg;
    pa.hlbg = P.hg ? at<float>(base, P.hlbg) : nullptr;
    pa.hgd = P.hg ? at<float>(base, P.hgd) : nullptr;
    pa.hperm = P.hg ? at<int>(base, P.hperm) : nullptr;
    pa.hgoff = P.hg ? at<int>(base, P.hgoff) : nullptr;
    pa.acc = P.acc ? at<long long>(base, P.acc) : nullptr;
    pa.accC = P.acc ? reinterpret_cast<int32_t*>(pa.acc + (size_t)K * d) : nullptr;

    FinArgs& fa = L.fa;
    memset(&fa, 0, sizeof(fa));
    fa.K = K;
    fa.d = d;
    fa.nb = P.nb;
    fa.part_f64 = L.f64;
    fa.pS = at<void>(base, P.pS);
    fa.pCnt = at<int32_t>(base, P.pCnt);
    fa.KB = P.KB;
    fa.C64 = at<double>(base, P.C64);
    fa.CAU = at<double>(base, P.CAU);
    fa.Fprev = at<double>(base, P.Fprev);
    fa.dF = at<double>(base, P.dF);
    fa.dG = at<double>(base, P.dG);
    fa.pDots = at<double>(base, P.pDots);
    fa.st = L.st;
    fa.m_max = L.m_max;
    fa.max_iter = p.max_iter;
    fa.lloyd_only = p.lloyd_only;
    fa.rank_tol = p.rank_tol;
    fa.ls_mode = ls_mode();
    fa.qrw = at<double>(base, P.qrw);
    fa.fuse_mix = fuse_mix_rule(K, d) ? 1 : 0;
    fa.part_fx = pa.acc ? 1 : 0;
    fa.acc = pa.acc;
    fa.accC = pa.accC;
    fa.DP = P.DP;
    fa.fp32_path = !L.f64;
    fa.origin = at<float>(base, P.origin);
    fa.cpk[0] = at<float>(base, P.cpk0);
    fa.cpk[1] = at<float>(base, P.cpk1);
    fa.c32[0] = at<float>(base, P.c32_0);
    fa.c32[1] = at<float>(base, P.c32_1);

    MixArgs& ma = L.ma;
    memset(&ma, 0, sizeof(ma));
    ma.K = K;
    ma.d = d;
    ma.Kpad = P.Kpad;
    ma.DP = P.DP;
    ma.fp32_path = !L.f64;
    ma.C64 = at<double>(base, P.C64);
    ma.CAU = at<double>(base, P.CAU);
    ma.dG = at<double>(base, P.dG);
    ma.m_max = L.m_max > 0 ? L.m_max : 1;
    ma.origin = at<float>(base, P.origin);
    ma.cpk[0] = at<float>(base, P.cpk0);
    ma.cpk[1] = at<float>(base, P.cpk1);
    ma.c32[0] = at<float>(base, P.c32_0);
    ma.c32[1] = at<float>(base, P.c32_1);
    ma.st = L.st;

    L.nsm = nsm;
    L.X32 = reinterpret_cast<const float*>(X->X);
    if (P.dense) {
        fa.part_fx = 2;                  // the update chain's int64 fixed-point totals
        fa.fxs_ptr = reinterpret_cast<const int*>(at<unsigned int>(base, P.counter) + 3);
        fa.fuse_mix = 0;
        fa.fp32_path = 0;
        ma.fp32_path = 0;                // the mix only writes C; the BF16 packing is separate
        DenseArgs& da = L.da;
        da = dense_args(base, P, L.X32, X->N, d, K);
        da.Xb = reinterpret_cast<const __nv_bfloat16*>(X->X_bf16);
        da.prescaled = 1;                // max ||x|| from the prologue's check fixes the update's scale
        const int im = dense_inc_mode();
        da.inc = im != 0;                // solver passes add only the rows whose label changed
        if (im == 2) da.inc_cap = -1;
        if (im == 3) da.inc_cap = X->N;
        fa.inc = da.inc;
        for (int i = 0; i < 2; ++i) {
            fa.Spair[i] = da.Spair[i];
            fa.Npair[i] = da.Npair[i];
        }
        da.thr = thr;
        da.lloyd_only = p.lloyd_only;
        da.fixed_m = p.fixed_m ? 1 : 0;
        da.eps1 = p.eps1;
        da.eps2 = p.eps2;
        da.m_max = L.m_max;
        da.max_iter = p.max_iter;
        L.pk = pack_args(base, P, d, K);
        L.pk.check_done = 1;
        L.xlo = dense_xlo(base, P, X);
        L.xsplit = X->X_bf16_lo == nullptr;
        L.maps_ok = dense_maps(base, P, X->X_bf16, L.xlo, X->N, d, &L.maps) &&
                    dense_maps(base, P, at<void>(base, P.xch), at<void>(base, P.xcl), X->N, d, &L.maps_c);
        L.dbounds = hamerly_mode();
        if (L.dbounds) {
            L.dmap = at<int>(base, P.map);
            L.dnrows = at<unsigned int>(base, P.nrows);
            L.dxch = at<void>(base, P.xch);
            L.dxcl = at<void>(base, P.xcl);
            da.hub = at<float>(base, P.hub);
            da.hlb = at<float>(base, P.hlb);
            da.xn2 = at<float>(base, P.xn2);
            da.hlast = at<float>(base, P.hlast);
            da.drift = at<float>(base, P.drift);
        }
    }
    return L;
}

// Capture of a conditional IF node inside a loop body that is being captured on a stream: the
// handle (value 0 at every graph launch) belongs to the body graph, the kernels captured before the
// node set it each iteration, and the chain inside the node is captured into the node's own graph.
struct IfCapture {
    cudaGraph_t body = nullptr;
    cudaGraphConditionalHandle h = 0;
};

cudaError_t if_handle(cudaStream_t s, IfCapture& c)
{
    cudaStreamCaptureStatus cs;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &c.body, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    return cudaGraphConditionalHandleCreate(&c.h, c.body, 0, cudaGraphCondAssignDefault);
}

// Runs the chain f launches inside an IF node on c.h that depends on everything s captured so far;
// the capture on s then resumes after the node.
template <typename F>
cudaError_t if_chain(cudaStream_t s, const IfCapture& c, F f)
{
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    cudaGraph_t tmp = nullptr;
    if ((e = cudaStreamEndCapture(s, &tmp)) != cudaSuccess) return e;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = c.h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t nif;
    if ((e = cudaGraphAddNode(&nif, c.body, dv.data(), nullptr, dv.size(), &cp)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCaptureToGraph(s, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
    const cudaError_t ef = f();
    e = cudaStreamEndCapture(s, &tmp);
    if (ef != cudaSuccess) return ef;
    if (e != cudaSuccess) return e;
    return cudaStreamBeginCaptureToGraph(s, c.body, &nif, nullptr, 1, cudaStreamCaptureModeRelaxed);
}

// One dense pass (assignment, rescoring, update chain with the controller) in the given mode.
cudaError_t dense_pass(const Launch& L, int mode, int use_cond, cudaGraphConditionalHandle h, cudaStream_t s,
                       bool assign = true, int use_rev = 0, cudaGraphConditionalHandle hr = 0)
{
    DenseArgs a = L.da;
    a.mode = mode;
    a.use_cond = use_cond;
    a.cond = h;
    a.use_cond_rev = use_rev;
    a.cond_rev = hr;
    cudaError_t e = cudaSuccess;
    const bool bounded = assign && L.dbounds && (mode == MODE_INIT || mode == MODE_TRIAL || mode == MODE_REVERT);
    if (!bounded) {
        a.hub = a.hlb = nullptr;
        if (assign) e = launch_dense_pass(a, L.maps, L.nsm, s);
    } else if (mode == MODE_INIT) {     // every row scanned; the bounds and the last centroids set
        e = launch_dense_bounds(a, nullptr, nullptr, nullptr, nullptr, L.nsm, s);
        if (e == cudaSuccess) e = launch_dense_pass(a, L.maps, L.nsm, s);
    } else {                            // the rows the bounds cannot keep, compacted
        a.map = L.dmap;
        a.nrows = L.dnrows;
        e = launch_dense_bounds(a, a.Xb, L.xlo, L.dxch, L.dxcl, L.nsm, s);
        if (e == cudaSuccess) e = launch_dense_pass(a, L.maps_c, L.nsm, s);
        a.map = nullptr;                // the update reads only the count (rows scanned, for the info)
    }
    if (e == cudaSuccess) e = launch_dense_update(a, L.P.nbk, L.P.max_chunks, s);
    return e;
}

// Prologue: C^0 -> P^0 -> G^0 = C^1 (Algorithm 1's first line).
cudaError_t launch_prologue(const Launch& L, cudaStream_t s, cudaGraphConditionalHandle h)
{
    if (L.P.dense) {
        cudaError_t e = cudaMemsetAsync(L.pa.counter, 0, 256, s);
        if (e == cudaSuccess)      // the fixed-point totals the update chain adds into
            e = cudaMemsetAsync(L.da.acc, 0, (size_t)L.K * L.d * 8 + (size_t)L.K * 4, s);
        if (e == cudaSuccess)
            e = launch_prep(L.C0, false, L.K, L.d, 0, 0, L.ma.C64, const_cast<float*>(L.ma.origin), nullptr, nullptr,
                            nullptr, L.st, L.p.m_init, L.m_max, s, 0);
        if (e == cudaSuccess)
            e = (L.da.inc && xcheck_blocks(L.nsm) > QX_BLOCKS)
                    ? cudaErrorInvalidConfiguration
                    : launch_xcheck(L.X32, L.N, L.d, L.da.counter + 4, const_cast<float*>(L.da.xn2), L.st, L.nsm, s,
                                    L.da.inc ? L.da.qx : nullptr, L.da.counter + 8);
        if (e == cudaSuccess && L.xsplit)
            e = launch_xsplit(L.X32, L.da.Xb, const_cast<void*>(L.xlo), L.N * (int64_t)L.d, L.nsm, s);
        PackArgs pk = L.pk;
        pk.nsets = 1;
        pk.check_done = 0;
        if (e == cudaSuccess) e = launch_pack_dense(pk, s);
        if (e == cudaSuccess) e = dense_pass(L, MODE_INIT, 0, h, s);
        FinArgs f = L.fa;
        f.mode = MODE_INIT;
        if (e == cudaSuccess) e = launch_fin(f, L.P.nfin, s);
        MixArgs m = L.ma;
        m.mode = MODE_INIT;
        if (e == cudaSuccess) e = launch_mix(m, s);
        pk = L.pk;
        pk.check_done = 0;
        if (e == cudaSuccess) e = launch_pack_dense(pk, s);
        return e;
    }
    cudaError_t e = cudaMemsetAsync(L.pa.counter, 0, 256, s);
    if (e == cudaSuccess)
        e = launch_prep(L.C0, L.f64, L.K, L.d, L.P.Kpad, L.P.DP, L.ma.C64, const_cast<float*>(L.ma.origin),
                        L.ma.cpk[0], L.ma.cpk[1], L.ma.c32[0], L.st, L.p.m_init, L.m_max, s);
    PassArgs a = L.pa;
    a.mode = MODE_INIT;
    a.flags = F_ASSIGN | F_BINS | F_ENERGY | F_CHECK;
    if (e == cudaSuccess && a.hg > 0) e = launch_groups(L.ma.C64, L.K, L.d, a.hg, a.hperm, a.hgoff, s);
    if (e == cudaSuccess && a.ham) e = launch_hprep(a, MODE_INIT, s);
    if (e == cudaSuccess) e = launch_pass_lowd(a, L.prec, L.d, L.P.nb, s);
    FinArgs f = L.fa;
    f.mode = MODE_INIT;
    if (e == cudaSuccess) e = launch_fin(f, L.P.nfin, s);
    if (!L.fa.fuse_mix) {
        MixArgs m = L.ma;
        m.mode = MODE_INIT;
        if (e == cudaSuccess) e = launch_mix(m, s);
    }
    (void)h;
    return e;
}

// One loop pass t of Algorithm 1 (or Lloyd): trial assignment + controller, conditional revert,
// update + history + least squares, accelerated iterate (which also ends the graph loop).
cudaError_t launch_body(const Launch& L, cudaStream_t s, int use_cond, cudaGraphConditionalHandle h)
{
    // Inside a graph the REVERT pass sits in an IF node that its TRIAL pass sets, so an accepted
    // accelerated iterate launches nothing for it; the REVERT kernels still check the flag.
    IfCapture ic;
    const char* ife = getenv("KM_REVERT_IF");         // 0: plain launches (the kernels return at once)
    const int lowd_if = ife ? (ife[0] == '1' || ife[0] == '3') : 0;
    const int dense_if = ife ? (ife[0] == '2' || ife[0] == '3') : 1;
    const int use_rev_if = L.P.dense ? dense_if : lowd_if;
    if (use_cond && use_rev_if) {
        const cudaError_t e = if_handle(s, ic);
        if (e != cudaSuccess) return e;
    }
    if (L.P.dense) {
        cudaError_t e = dense_pass(L, MODE_TRIAL, use_cond, h, s, true, use_cond && use_rev_if, ic.h);
        if (e == cudaSuccess) {
            auto rev = [&]() { return dense_pass(L, MODE_REVERT, use_cond, h, s); };
            e = use_cond && use_rev_if ? if_chain(s, ic, rev) : rev();
        }
        FinArgs f = L.fa;
        f.mode = MODE_TRIAL;
        f.use_cond = use_cond;
        f.cond = h;
        if (e == cudaSuccess) e = launch_fin(f, L.P.nfin, s);
        MixArgs m = L.ma;
        m.mode = MODE_TRIAL;
        if (e == cudaSuccess) e = launch_mix(m, s);
        if (e == cudaSuccess) e = launch_pack_dense(L.pk, s);
        return e;
    }
    PassArgs a = L.pa;
    a.mode = MODE_TRIAL;
    a.flags = F_ASSIGN | F_BINS | F_ENERGY | F_CHANGED;
    a.use_cond = use_cond;
    a.cond = h;
    a.use_cond_rev = use_cond && use_rev_if;
    a.cond_rev = ic.h;
    cudaError_t e = a.ham ? launch_hprep(a, MODE_TRIAL, s) : cudaSuccess;
    if (e == cudaSuccess) e = launch_pass_lowd(a, L.prec, L.d, L.P.nb, s);
    a.mode = MODE_REVERT;       // its bound inputs come from the TRIAL pass's last block
    a.use_cond_rev = 0;
    if (e == cudaSuccess) {
        auto rev = [&]() { return launch_pass_lowd(a, L.prec, L.d, L.P.nb, s); };
        e = use_cond && use_rev_if ? if_chain(s, ic, rev) : rev();
    }
    FinArgs f = L.fa;
    f.mode = MODE_TRIAL;
    f.use_cond = use_cond;
    f.cond = h;
    if (e == cudaSuccess) e = launch_fin(f, L.P.nfin, s);
    if (!L.fa.fuse_mix) {
        MixArgs m = L.ma;
        m.mode = MODE_TRIAL;
        if (e == cudaSuccess) e = launch_mix(m, s);
    }
    return e;
}

// Epilogue: the energy of (P^t, G^t) if the loop stopped at max_iter, results and info.
cudaError_t launch_epilogue(const Launch& L, cudaStream_t s)
{
    cudaError_t e;
    if (L.P.dense) {
        e = dense_pass(L, MODE_EPI, 0, 0, s, false);
    } else {
        PassArgs a = L.pa;
        a.mode = MODE_EPI;
        a.flags = F_ENERGY;
        e = launch_pass_lowd(a, L.prec, L.d, L.P.nb, s);
    }
    if (e == cudaSuccess)
        e = launch_epi(L.f64, L.st, L.ma.C64, L.ma.CAU, L.C_out, (size_t)L.K * L.d, L.rhoA, L.rhoB, L.rho_out, L.N,
                       L.info, s);
    return e;
}

// KM_GRAPH=0 in the environment launches the same kernels from a host loop (one wait per
// iteration) instead of the graph; profilers cannot see kernels inside conditional graphs.
bool graph_mode()
{
    const char* v = getenv("KM_GRAPH");
    return !(v && v[0] == '0');
}

struct DevInfoH {
    int iters, accepted, rejected, passes, converged, m_final, status, ls_qr;
    double E;
    long long rescored;
    long long scanned;
};

kmeans_status validate_params(kmeans_ctx* ctx, const kmeans_params& p)
{
    if (p.m_max < 0 || p.m_max > MMAX) return fail(ctx, KM_EINVAL, "m_max must be in [0, 32]");
    if (p.max_iter < 1) return fail(ctx, KM_EINVAL, "max_iter must be >= 1");
    if (!(p.tol >= 0.0)) return fail(ctx, KM_EINVAL, "tol must be >= 0");
    if (!(p.rank_tol >= 0.0)) return fail(ctx, KM_EINVAL, "rank_tol must be >= 0");
    return KM_OK;
}

// Once-per-solve setup and result-copy arguments of one low-d solve (batched and serving paths).
PrepArgs prep_args(const Launch& L, int m_init)
{
    PrepArgs pp;
    memset(&pp, 0, sizeof(pp));
    pp.C0 = L.C0;
    pp.f64 = L.f64;
    pp.K = L.K;
    pp.d = L.d;
    pp.Kpad = L.P.Kpad;
    pp.DP = L.P.DP;
    pp.pack = 1;
    pp.C64 = L.ma.C64;
    pp.origin = const_cast<float*>(L.ma.origin);
    pp.cpk0 = L.ma.cpk[0];
    pp.cpk1 = L.ma.cpk[1];
    pp.c32_0 = L.ma.c32[0];
    pp.st = L.st;
    pp.m_init = m_init;
    pp.m_max = L.m_max;
    pp.counter = L.pa.counter;
    return pp;
}

int epi_blocks(int64_t N, size_t n)
{
    const int64_t big = std::max<int64_t>(N, (int64_t)n);
    return (int)std::min<int64_t>(64, (big + 2047) / 2048);
}

EpiArgs epi_args(const Launch& L, void* info)
{
    EpiArgs ea;
    memset(&ea, 0, sizeof(ea));
    ea.f64 = L.f64;
    ea.st = L.st;
    ea.C64 = L.ma.C64;
    ea.CAU = L.ma.CAU;
    ea.C_out = L.C_out;
    ea.n = (size_t)L.K * L.d;
    ea.rhoA = L.rhoA;
    ea.rhoB = L.rhoB;
    ea.rho_out = L.rho_out;
    ea.N = L.N;
    ea.info = info;
    ea.nblk = epi_blocks(L.N, ea.n);
    return ea;
}

// Work items of the mix kernel of a low-d solve (none when the accelerated iterate is fused).
int mix_blocks(int K, int d) { return fuse_mix_rule(K, d) ? 0 : (K * 32 + 255) / 256; }

void fill_info(kmeans_info* info, const DevInfoH* di, float ms)
{
    info->iters = di->iters;
    info->accepted = di->accepted;
    info->rejected = di->rejected;
    info->assign_passes = di->passes;
    info->converged = di->converged;
    info->m_final = di->m_final;
    info->E = di->E;
    info->rescored_rows = di->rescored;
    info->device_ms = ms;
    info->status = di->status;
    info->ls_qr_solves = di->ls_qr;
    info->scanned_rows = di->scanned;
}

// Add  prologue -> while (cond) { body } -> epilogue  to graph g as an independent chain.  The
// prologue and the epilogue are captured into child graphs, the body straight into the conditional
// node's body graph; the body's kernels end the loop with cudaGraphSetConditional(h, 0).
template <typename Pro, typename Body, typename Epi>
kmeans_status add_while_chain(kmeans_ctx* ctx, cudaGraph_t g, Pro pro, Body body, Epi epi)
{
    cudaGraph_t gp = nullptr, ge = nullptr;
    cudaGraphConditionalHandle h;
    KM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));

    KM_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = pro(ctx->cap);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &gp);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "prologue launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "prologue capture");
    }
    cudaGraphNode_t np, nc, ne;
    KM_CUDA(cudaGraphAddChildGraphNode(&np, g, nullptr, 0, gp));

    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    KM_CUDA(cudaGraphAddNode(&nc, g, &np, nullptr, 1, &cp));
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    KM_CUDA(cudaStreamBeginCaptureToGraph(ctx->cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = body(ctx->cap, h);
        cudaGraph_t bout = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &bout);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "loop body launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "loop body capture");
    }

    KM_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = epi(ctx->cap);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &ge);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "epilogue launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "epilogue capture");
    }
    KM_CUDA(cudaGraphAddChildGraphNode(&ne, g, &nc, 1, ge));
    cudaGraphDestroy(gp);
    cudaGraphDestroy(ge);
    return KM_OK;
}

// One executable graph holding one such chain.
template <typename Pro, typename Body, typename Epi>
kmeans_status record_while_graph(kmeans_ctx* ctx, Pro pro, Body body, Epi epi, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    KM_CUDA(cudaGraphCreate(&g, 0));
    kmeans_status s = add_while_chain(ctx, g, pro, body, epi);
    if (s == KM_OK) {
        cudaError_t e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    cudaGraphDestroy(g);
    return s;
}

}  // namespace
