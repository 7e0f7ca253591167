// C ABI of libkmeans_aa (declared in include/kmeans_aa.h): context, workspace, the standalone
// assignment / update / energy calls, and the solver, which runs every iteration of Lloyd or
// Algorithm 1 inside one CUDA graph:
//
//   prologue : k_prep -> pass(INIT: P^0 = Assign(C^0)) -> k_fin(INIT: G^0, F^0) -> k_mix(INIT: C^1)
//   while    : pass(TRIAL) -> pass(REVERT, exits at once unless the safeguard fired)
//              -> k_fin(update, history, Gram, theta) -> k_mix(C^{t+1}; ends the loop when done)
//   epilogue : pass(EPI: energy if stopped at max_iter) -> k_epi(results, info)
//
// All per-iteration decisions stay on the device; the host waits once per solve.
#include "dense.cuh"
#include "km_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

using namespace km;

namespace {

struct GraphKey {
    const void* X;
    const void* Xb;
    int64_t N;
    int d, K, prec;
    const void* C0;
    void* C_out;
    int32_t* rho_out;
    kmeans_params p;
    void* arena;
    size_t arena_bytes;
};

struct Plan {
    // offsets into the arena
    size_t st, rhoA, rhoB, C64, CAU, Fprev, dF, dG, cpk0, cpk1, c32_0, c32_1, origin;
    size_t pS, pCnt, pE, pNch, pResc, pBad, pDots, counter, info;
    size_t hX, hXb, hC0, hCout, hRho;   // device copies for kmeans_solve_host
    // dense path (tensor-core assignment, sort-based update)
    size_t cb0, cb1, cn0, cn1, xnorm, queue, qcount, err, hist, counts, off, choff, chunk_cluster, nchunks, perm,
        part, pe, pnch, S, rowe, rown;
    size_t total;
    int nb, nfin, KB, Kpad, DP;
    bool dense;
    int dpad, nbk, rpb, max_chunks;
    size_t smem;
};

constexpr int DENSE_RPB = 4096;   // rows per block of the dense update's histogram and scatter
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
    return KM_OK;
}

int pass_blocks(kmeans_ctx* ctx, int64_t N, size_t smem)
{
    int per_sm = (int)((200 * 1024) / (smem + 2048));
    if (per_sm > 2) per_sm = 2;           // register-limited: 256 threads x ~128 registers
    if (per_sm < 1) per_sm = 1;
    int64_t nb = (int64_t)ctx->nsm * per_sm;
    const int64_t need = (N + LOWD_THREADS - 1) / LOWD_THREADS;
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
    P.rpb = DENSE_RPB;
    P.nbk = (int)((N + DENSE_RPB - 1) / DENSE_RPB);
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
    P.cpk0 = P.cpk1 = 0;
    P.c32_0 = take(n * 4);
    P.c32_1 = take(n * 4);
    P.origin = take(256);
    P.cb0 = take((size_t)P.Kpad * P.dpad * 2);
    P.cb1 = take((size_t)P.Kpad * P.dpad * 2);
    P.cn0 = take((size_t)P.Kpad * 4);
    P.cn1 = take((size_t)P.Kpad * 4);
    P.xnorm = take((size_t)N * 4);
    P.queue = take((size_t)N * 4 * 4);   // full-rescore rows, then (row, i1, i2) candidate pairs
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
    P.S = take(n * 8);
    P.rowe = take(4096 * 8);
    P.rown = take(4096 * 8);
    P.pS = P.S;
    P.pCnt = P.counts;
    P.pE = P.pNch = P.pResc = P.pBad = 0;
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

kmeans_status make_plan(kmeans_ctx* ctx, int64_t N, int d, int K, int prec, int m_max, bool host_copies,
                        Plan& P, bool bins = true)
{
    P.dense = false;
    P.dpad = P.nbk = P.rpb = P.max_chunks = 0;
    if (prec == KM_BF16_F32 && d > 16) return make_plan_dense(ctx, N, d, K, m_max, host_copies, P);
    if (d > 16) return fail(ctx, KM_EINVAL, "d > 16 needs KM_BF16_F32 (the tensor-core path)");
    const bool f32 = prec != KM_F64;
    const size_t esz = f32 ? 4 : 8;
    P.DP = pass_lowd_dp(d);
    P.Kpad = (K + CH - 1) / CH * CH;
    P.smem = pass_lowd_smem(prec, d, K, P.Kpad, bins);
    if (P.smem > 200 * 1024)
        return fail(ctx, KM_EINVAL, bins ? "K*d too large for the fused low-d update" : "K*d too large");
    P.nb = pass_blocks(ctx, N, P.smem);
    P.nfin = fin_blocks(K, d, &P.KB);
    const size_t n = (size_t)K * d;
    const int mm = m_max > 0 ? m_max : 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    P.counter = take(256);          // fixed offset 0 for every plan; zeroed at the start of every call
    P.st = take(sizeof(SolveState));
    P.rhoA = take((size_t)N * 4);
    P.rhoB = take((size_t)N * 4);
    P.C64 = take(n * 8);
    P.CAU = take(n * 8);
    P.Fprev = take(n * 8);
    P.dF = take((size_t)mm * n * 8);
    P.dG = take((size_t)mm * n * 8);
    P.cpk0 = take((size_t)P.Kpad * P.DP * 4);
    P.cpk1 = take((size_t)P.Kpad * P.DP * 4);
    P.c32_0 = take(n * 4);
    P.c32_1 = take(n * 4);
    P.origin = take(64 * 4);
    P.pS = take((size_t)P.nb * n * esz);
    P.pCnt = take((size_t)P.nb * K * 4);
    P.pE = take((size_t)P.nb * 8);
    P.pNch = take((size_t)P.nb * 8);
    P.pResc = take((size_t)P.nb * 8);
    P.pBad = take((size_t)P.nb * 4);
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
T* at(kmeans_ctx* ctx, size_t off)
{
    return reinterpret_cast<T*>(static_cast<char*>(ctx->arena) + off);
}

PassArgs base_pass(kmeans_ctx* ctx, const Plan& P, const void* X, int64_t N, int K, int prec)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.X = X;
    a.N = N;
    a.K = K;
    a.Kpad = P.Kpad;
    a.cpk[0] = at<float>(ctx, P.cpk0);
    a.cpk[1] = at<float>(ctx, P.cpk1);
    a.c32[0] = at<float>(ctx, P.c32_0);
    a.c32[1] = at<float>(ctx, P.c32_1);
    a.c64[0] = at<double>(ctx, P.C64);
    a.c64[1] = at<double>(ctx, P.CAU);
    a.origin = at<float>(ctx, P.origin);
    a.rho[0] = at<int32_t>(ctx, P.rhoA);
    a.rho[1] = at<int32_t>(ctx, P.rhoB);
    a.pS = at<void>(ctx, P.pS);
    a.pCnt = at<int32_t>(ctx, P.pCnt);
    a.pE = at<double>(ctx, P.pE);
    a.pNch = at<long long>(ctx, P.pNch);
    a.pResc = at<long long>(ctx, P.pResc);
    a.pBad = at<int>(ctx, P.pBad);
    a.counter = at<unsigned int>(ctx, P.counter);
    a.st = at<SolveState>(ctx, P.st);
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
    alignas(64) unsigned char tmX[128];
    alignas(64) unsigned char tmC0[128];
    alignas(64) unsigned char tmC1[128];
    bool maps_ok = true;
};

// Dense-path arguments over the plan's buffers (centroid sets 0 = C^t, 1 = C_AU).
DenseArgs dense_args(kmeans_ctx* ctx, const Plan& P, const float* X32, int64_t N, int d, int K)
{
    DenseArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N;
    a.d = d;
    a.dpad = P.dpad;
    a.K = K;
    a.Kpad = P.Kpad;
    a.X = X32;
    a.xnorm = at<float>(ctx, P.xnorm);
    a.cn[0] = at<float>(ctx, P.cn0);
    a.cn[1] = at<float>(ctx, P.cn1);
    a.c32[0] = at<float>(ctx, P.c32_0);
    a.c32[1] = at<float>(ctx, P.c32_1);
    a.c64[0] = at<double>(ctx, P.C64);
    a.c64[1] = at<double>(ctx, P.CAU);
    // BF16 score error bound: 2 (2 u_b + d u) |x| max|c| for 2 x.c, u max|c|^2 for ||c||^2, with a
    // factor 2 of allowance for the accumulation order inside the MMA
    const double ub = 1.0 / 512.0, u = 5.9604644775390625e-8;
    a.bcoef_a = (float)(2.0 * (2.0 * (2.0 * ub + d * u)) * (1.0 + 2.0 * ub));
    a.bcoef_b = (float)(2.0 * 2.0 * u);
    a.rho_pair[0] = at<int32_t>(ctx, P.rhoA);
    a.rho_pair[1] = at<int32_t>(ctx, P.rhoB);
    a.queue = at<int>(ctx, P.queue);
    a.cand = at<int>(ctx, P.queue) + N;
    a.qcount = at<unsigned int>(ctx, P.qcount);
    a.err = at<int>(ctx, P.err);
    a.rows_per_block = P.rpb;
    a.hist = at<int>(ctx, P.hist);
    a.counts = at<int32_t>(ctx, P.counts);
    a.off = at<int>(ctx, P.off);
    a.choff = at<int>(ctx, P.choff);
    a.chunk_cluster = at<int>(ctx, P.chunk_cluster);
    a.nchunks = at<int>(ctx, P.nchunks);
    a.perm = at<int>(ctx, P.perm);
    a.part = at<float>(ctx, P.part);
    a.pe = at<double>(ctx, P.pe);
    a.pnch = at<long long>(ctx, P.pnch);
    a.S = at<double>(ctx, P.S);
    a.counter = at<unsigned int>(ctx, P.counter);
    a.st = at<SolveState>(ctx, P.st);
    return a;
}

PackArgs pack_args(kmeans_ctx* ctx, const Plan& P, int d, int K)
{
    PackArgs p;
    memset(&p, 0, sizeof(p));
    p.K = K;
    p.Kpad = P.Kpad;
    p.d = d;
    p.dpad = P.dpad;
    p.nsets = 2;
    p.src64[0] = at<double>(ctx, P.C64);
    p.src64[1] = at<double>(ctx, P.CAU);
    p.cb[0] = at<__nv_bfloat16>(ctx, P.cb0);
    p.cb[1] = at<__nv_bfloat16>(ctx, P.cb1);
    p.cn[0] = at<float>(ctx, P.cn0);
    p.cn[1] = at<float>(ctx, P.cn1);
    p.c32[0] = at<float>(ctx, P.c32_0);
    p.c32[1] = at<float>(ctx, P.c32_1);
    p.st = at<SolveState>(ctx, P.st);
    return p;
}

bool dense_maps(kmeans_ctx* ctx, const Plan& P, const void* Xb, int64_t N, int d, void* tmX, void* tmC0, void* tmC1)
{
    return make_tmap_bf16(tmX, Xb, N, d, 128) &&
           make_tmap_bf16(tmC0, at<void>(ctx, P.cb0), P.Kpad, P.dpad, 256) &&
           make_tmap_bf16(tmC1, at<void>(ctx, P.cb1), P.Kpad, P.dpad, 256);
}

Launch make_launch(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, int K, const void* C0,
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
    L.st = at<SolveState>(ctx, P.st);
    L.info = at<void>(ctx, P.info);
    L.rhoA = at<int32_t>(ctx, P.rhoA);
    L.rhoB = at<int32_t>(ctx, P.rhoB);
    const int d = X->d;
    const int64_t thr = p.tol > 0 ? (int64_t)(p.tol * (double)X->N) : 0;

    PassArgs& pa = L.pa;
    pa = base_pass(ctx, P, X->X, X->N, K, X->prec);
    set_bound(pa, d);
    pa.m_max = L.m_max;
    pa.max_iter = p.max_iter;
    pa.lloyd_only = p.lloyd_only;
    pa.eps1 = p.eps1;
    pa.eps2 = p.eps2;
    pa.thr = thr;

    FinArgs& fa = L.fa;
    memset(&fa, 0, sizeof(fa));
    fa.K = K;
    fa.d = d;
    fa.nb = P.nb;
    fa.part_f64 = L.f64;
    fa.pS = at<void>(ctx, P.pS);
    fa.pCnt = at<int32_t>(ctx, P.pCnt);
    fa.KB = P.KB;
    fa.C64 = at<double>(ctx, P.C64);
    fa.CAU = at<double>(ctx, P.CAU);
    fa.Fprev = at<double>(ctx, P.Fprev);
    fa.dF = at<double>(ctx, P.dF);
    fa.dG = at<double>(ctx, P.dG);
    fa.pDots = at<double>(ctx, P.pDots);
    fa.st = L.st;
    fa.m_max = L.m_max;
    fa.max_iter = p.max_iter;
    fa.lloyd_only = p.lloyd_only;
    fa.rank_tol = p.rank_tol;
    fa.fuse_mix = (K <= 1024 && (size_t)K * d <= 16384) ? 1 : 0;
    fa.DP = P.DP;
    fa.fp32_path = !L.f64;
    fa.origin = at<float>(ctx, P.origin);
    fa.cpk[0] = at<float>(ctx, P.cpk0);
    fa.cpk[1] = at<float>(ctx, P.cpk1);
    fa.c32[0] = at<float>(ctx, P.c32_0);
    fa.c32[1] = at<float>(ctx, P.c32_1);

    MixArgs& ma = L.ma;
    memset(&ma, 0, sizeof(ma));
    ma.K = K;
    ma.d = d;
    ma.Kpad = P.Kpad;
    ma.DP = P.DP;
    ma.fp32_path = !L.f64;
    ma.C64 = at<double>(ctx, P.C64);
    ma.CAU = at<double>(ctx, P.CAU);
    ma.dG = at<double>(ctx, P.dG);
    ma.m_max = L.m_max > 0 ? L.m_max : 1;
    ma.origin = at<float>(ctx, P.origin);
    ma.cpk[0] = at<float>(ctx, P.cpk0);
    ma.cpk[1] = at<float>(ctx, P.cpk1);
    ma.c32[0] = at<float>(ctx, P.c32_0);
    ma.c32[1] = at<float>(ctx, P.c32_1);
    ma.st = L.st;

    L.nsm = ctx->nsm;
    L.X32 = reinterpret_cast<const float*>(X->X);
    if (P.dense) {
        fa.part_f64 = 1;                 // S: FP64 residual sums per cluster, one "partial block"
        fa.fuse_mix = 0;
        fa.fp32_path = 0;
        ma.fp32_path = 0;                // the mix only writes C; the BF16 packing is separate
        DenseArgs& da = L.da;
        da = dense_args(ctx, P, L.X32, X->N, d, K);
        da.Xb = reinterpret_cast<const __nv_bfloat16*>(X->X_bf16);
        da.thr = thr;
        da.lloyd_only = p.lloyd_only;
        da.eps1 = p.eps1;
        da.eps2 = p.eps2;
        da.m_max = L.m_max;
        da.max_iter = p.max_iter;
        L.pk = pack_args(ctx, P, d, K);
        L.pk.check_done = 1;
        L.maps_ok = dense_maps(ctx, P, X->X_bf16, X->N, d, L.tmX, L.tmC0, L.tmC1);
    }
    return L;
}

// One dense pass (assignment, rescoring, update chain with the controller) in the given mode.
cudaError_t dense_pass(const Launch& L, int mode, int use_cond, cudaGraphConditionalHandle h, cudaStream_t s,
                       bool assign = true)
{
    DenseArgs a = L.da;
    a.mode = mode;
    a.use_cond = use_cond;
    a.cond = h;
    cudaError_t e = cudaSuccess;
    if (assign) e = launch_dense_pass(a, L.tmX, L.tmC0, L.tmC1, L.nsm, s);
    if (e == cudaSuccess) e = launch_dense_update(a, L.P.nbk, L.P.max_chunks, s);
    return e;
}

// Prologue: C^0 -> P^0 -> G^0 = C^1 (Algorithm 1's first line).
cudaError_t launch_prologue(const Launch& L, cudaStream_t s, cudaGraphConditionalHandle h)
{
    if (L.P.dense) {
        cudaError_t e = cudaMemsetAsync(L.pa.counter, 0, 256, s);
        if (e == cudaSuccess)
            e = launch_prep(L.C0, false, L.K, L.d, 0, 0, L.ma.C64, const_cast<float*>(L.ma.origin), nullptr, nullptr,
                            nullptr, L.st, L.p.m_init, L.m_max, s, 0);
        if (e == cudaSuccess) e = launch_xnorm(L.X32, L.N, L.d, const_cast<float*>(L.da.xnorm), L.st, L.nsm, s);
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
    if (L.P.dense) {
        cudaError_t e = dense_pass(L, MODE_TRIAL, use_cond, h, s);
        if (e == cudaSuccess) e = dense_pass(L, MODE_REVERT, use_cond, h, s);
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
    cudaError_t e = launch_pass_lowd(a, L.prec, L.d, L.P.nb, s);
    a.mode = MODE_REVERT;
    if (e == cudaSuccess) e = launch_pass_lowd(a, L.prec, L.d, L.P.nb, s);
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

kmeans_status record_graph(kmeans_ctx* ctx, const Launch& L)
{
    cudaGraph_t g = nullptr, gp = nullptr, ge = nullptr;
    cudaGraphConditionalHandle h;
    KM_CUDA(cudaGraphCreate(&g, 0));
    KM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));

    KM_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = launch_prologue(L, ctx->cap, h);
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
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    KM_CUDA(cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = launch_body(L, ctx->cap, 1, h);
        cudaGraph_t bout = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &bout);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "loop body launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "loop body capture");
    }

    KM_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t e = launch_epilogue(L, ctx->cap);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &ge);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "epilogue launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "epilogue capture");
    }
    KM_CUDA(cudaGraphAddChildGraphNode(&ne, g, &nc, 1, ge));
    cudaGraphExec_t exec;
    KM_CUDA(cudaGraphInstantiate(&exec, g, 0));
    cudaGraphDestroy(gp);
    cudaGraphDestroy(ge);
    cudaGraphDestroy(g);
    if (ctx->have_graph) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = exec;
    ctx->have_graph = true;
    return KM_OK;
}

// KM_GRAPH=0 in the environment launches the same kernels from a host loop (one wait per
// iteration) instead of the graph; profilers cannot see kernels inside conditional graphs.
bool graph_mode()
{
    const char* v = getenv("KM_GRAPH");
    return !(v && v[0] == '0');
}

kmeans_status run_host_loop(kmeans_ctx* ctx, const Launch& L)
{
    cudaGraphConditionalHandle h = 0;
    KM_CUDA(launch_prologue(L, ctx->stream, h));
    int* done = reinterpret_cast<int*>(static_cast<char*>(ctx->h_info) + 128);
    for (int it = 0; it < L.p.max_iter + 2; ++it) {
        KM_CUDA(launch_body(L, ctx->stream, 0, h));
        KM_CUDA(cudaMemcpyAsync(done, &L.st->done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        KM_CUDA(cudaStreamSynchronize(ctx->stream));
        if (*done) break;
    }
    KM_CUDA(launch_epilogue(L, ctx->stream));
    return KM_OK;
}

struct DevInfoH {
    int iters, accepted, rejected, passes, converged, m_final, status, pad;
    double E;
    long long rescored;
};

kmeans_status validate_params(kmeans_ctx* ctx, const kmeans_params& p)
{
    if (p.m_max < 0 || p.m_max > MMAX) return fail(ctx, KM_EINVAL, "m_max must be in [0, 32]");
    if (p.max_iter < 1) return fail(ctx, KM_EINVAL, "max_iter must be >= 1");
    if (!(p.tol >= 0.0)) return fail(ctx, KM_EINVAL, "tol must be >= 0");
    if (!(p.rank_tol >= 0.0)) return fail(ctx, KM_EINVAL, "rank_tol must be >= 0");
    return KM_OK;
}

kmeans_status solve_device(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                           const kmeans_params& p, void* C_out, int32_t* rho_out, kmeans_info* info,
                           const Plan& P)
{
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.X = X->X;
    key.Xb = X->X_bf16;
    key.N = X->N;
    key.d = X->d;
    key.K = K;
    key.prec = X->prec;
    key.C0 = C0;
    key.C_out = C_out;
    key.rho_out = rho_out;
    key.p = p;
    key.arena = ctx->arena;
    key.arena_bytes = ctx->arena_bytes;
    const Launch L = make_launch(ctx, P, X, K, C0, p, C_out, rho_out);
    if (!L.maps_ok) return fail(ctx, KM_ECUDA, "cuTensorMapEncodeTiled failed (X_bf16 must be 16-byte aligned)");
    const bool use_graph = graph_mode();
    if (use_graph && (!ctx->have_graph || memcmp(&key, &ctx->key, sizeof(key)) != 0)) {
        kmeans_status s = record_graph(ctx, L);
        if (s != KM_OK) return s;
        ctx->key = key;
    }
    KM_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
    if (use_graph) {
        KM_CUDA(cudaGraphLaunch(ctx->exec, ctx->stream));
    } else {
        kmeans_status s = run_host_loop(ctx, L);
        if (s != KM_OK) return s;
    }
    KM_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
    KM_CUDA(cudaMemcpyAsync(ctx->h_info, at<void>(ctx, P.info), sizeof(DevInfoH), cudaMemcpyDeviceToHost,
                            ctx->stream));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    const DevInfoH* di = reinterpret_cast<const DevInfoH*>(ctx->h_info);
    if (info) {
        info->iters = di->iters;
        info->accepted = di->accepted;
        info->rejected = di->rejected;
        info->assign_passes = di->passes;
        info->converged = di->converged;
        info->m_final = di->m_final;
        info->E = di->E;
        info->rescored_rows = di->rescored;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        info->device_ms = ms;
    }
    if (di->status == KM_ENONFINITE) return fail(ctx, KM_ENONFINITE, "X contains NaN or Inf");
    if (di->status == KM_ETIMEOUT) return fail(ctx, KM_ETIMEOUT, "iteration guard tripped");
    return KM_OK;
}

// ---- standalone calls on the dense path
kmeans_status dense_pack_user(kmeans_ctx* ctx, const Plan& P, const void* C, int d, int K)
{
    PackArgs pk = pack_args(ctx, P, d, K);
    pk.nsets = 1;
    pk.src64[0] = nullptr;
    pk.src32 = reinterpret_cast<const float*>(C);
    pk.st = nullptr;
    pk.check_done = 0;
    KM_CUDA(launch_pack_dense(pk, ctx->stream));
    return KM_OK;
}

int rowred_blocks(kmeans_ctx* ctx) { return ctx->nsm * 4 < 4096 ? ctx->nsm * 4 : 4096; }

kmeans_status dense_assign_call(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, const void* C, int K,
                                int32_t* rho, const int32_t* rho_prev, int64_t* n_changed, void* dmin)
{
    kmeans_status s = ensure_arena(ctx, P.total);
    if (s != KM_OK) return s;
    const float* X32 = reinterpret_cast<const float*>(X->X);
    DenseArgs a = dense_args(ctx, P, X32, X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.Xb = reinterpret_cast<const __nv_bfloat16*>(X->X_bf16);
    a.rho_out = rho;
    a.rho_prev = rho_prev;
    a.out_nch = reinterpret_cast<long long*>(n_changed);
    alignas(64) unsigned char tmX[128], tmC[128], tmC1[128];
    if (!dense_maps(ctx, P, X->X_bf16, X->N, X->d, tmX, tmC, tmC1))
        return fail(ctx, KM_ECUDA, "cuTensorMapEncodeTiled failed (X_bf16 must be 16-byte aligned)");
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_dense_pass(a, tmX, tmC, tmC, ctx->nsm, ctx->stream));
    if (n_changed || dmin)
        KM_CUDA(launch_drow(a, rho, reinterpret_cast<float*>(dmin), at<double>(ctx, P.rowe), at<long long>(ctx, P.rown),
                            rowred_blocks(ctx), ctx->stream));
    return KM_OK;
}

kmeans_status dense_energy_call(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, const void* C, int K,
                                const int32_t* rho, double* E)
{
    kmeans_status s;
    DenseArgs a = dense_args(ctx, P, reinterpret_cast<const float*>(X->X), X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.out_E = E;
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_drow(a, rho, nullptr, at<double>(ctx, P.rowe), at<long long>(ctx, P.rown), rowred_blocks(ctx),
                        ctx->stream));
    return KM_OK;
}

kmeans_status dense_update_call(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, const int32_t* rho, int K,
                                const void* C_prev, void* C_out, int64_t* counts)
{
    kmeans_status s;
    DenseArgs a = dense_args(ctx, P, reinterpret_cast<const float*>(X->X), X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.rho_out = const_cast<int32_t*>(rho);     // read-only here: the labels of the update
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C_prev, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_dense_update(a, P.nbk, P.max_chunks, ctx->stream));
    FinArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = MODE_STANDALONE;
    f.K = K;
    f.d = X->d;
    f.nb = 1;
    f.part_f64 = 1;
    f.pS = a.S;
    f.pCnt = a.counts;
    f.KB = P.KB;
    f.C_ref = C_prev;
    f.C_out = C_out;
    f.out_f64 = 0;
    f.counts = counts;
    f.st = a.st;
    KM_CUDA(launch_fin(f, P.nfin, ctx->stream));
    return KM_OK;
}

}  // namespace

extern "C" {

void kmeans_default_params(kmeans_params* p)
{
    if (!p) return;
    p->m_max = 10;
    p->m_init = 2;
    p->max_iter = 1000;
    p->lloyd_only = 0;
    p->eps1 = 0.02;
    p->eps2 = 0.5;
    p->tol = 0.0;
    p->rank_tol = 1e-6;
}

const char* kmeans_status_string(kmeans_status s)
{
    switch (s) {
        case KM_OK: return "KM_OK";
        case KM_EINVAL: return "KM_EINVAL";
        case KM_ENOMEM: return "KM_ENOMEM";
        case KM_ECUDA: return "KM_ECUDA";
        case KM_ETIMEOUT: return "KM_ETIMEOUT";
        case KM_ENONFINITE: return "KM_ENONFINITE";
        case KM_EBUSY: return "KM_EBUSY";
    }
    return "KM_UNKNOWN";
}

const char* kmeans_last_error(const kmeans_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "";
}

kmeans_status kmeans_create(kmeans_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream)
{
    if (!out) return KM_EINVAL;
    *out = nullptr;
    kmeans_ctx* ctx = new kmeans_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc(&ctx->h_info, 256, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return KM_ECUDA;
    }
    *out = ctx;
    return KM_OK;
}

kmeans_status kmeans_destroy(kmeans_ctx* ctx)
{
    if (!ctx) return KM_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->have_graph) cudaGraphExecDestroy(ctx->exec);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->h_info) cudaFreeHost(ctx->h_info);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
    return KM_OK;
}

kmeans_status kmeans_set_stream(kmeans_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return KM_EINVAL;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return KM_OK;
}

size_t kmeans_workspace_bytes(const kmeans_ctx* ctx)
{
    return ctx ? ctx->arena_bytes : 0;
}

kmeans_status kmeans_assign(kmeans_ctx* ctx, const kmeans_data* X, const void* C, int32_t K, int32_t* rho,
                            const int32_t* rho_prev, int64_t* n_changed, void* dmin)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, true);
    if (s != KM_OK) return s;
    if (!C || !rho) return fail(ctx, KM_EINVAL, "C and rho must not be NULL");
    if (n_changed && !rho_prev) return fail(ctx, KM_EINVAL, "n_changed needs rho_prev");
    KM_CUDA(cudaSetDevice(ctx->device));
    Plan P;
    if ((s = make_plan(ctx, X->N, X->d, K, X->prec, 0, false, P, false)) != KM_OK) return s;
    if (P.dense) return dense_assign_call(ctx, P, X, C, K, rho, rho_prev, n_changed, dmin);
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    PassArgs a = base_pass(ctx, P, X->X, X->N, K, X->prec);
    a.mode = MODE_STANDALONE;
    a.flags = F_ASSIGN | (n_changed ? F_CHANGED : 0) | (dmin ? F_DMIN : 0) | (X->prec != KM_F64 ? F_PACK : 0);
    set_bound(a, X->d);
    if (X->prec == KM_F64) a.c64[0] = reinterpret_cast<const double*>(C);
    else a.rawC = reinterpret_cast<const float*>(C);
    a.rho[0] = rho;
    a.rho_prev = rho_prev;
    a.out_nch = reinterpret_cast<long long*>(n_changed);
    a.dmin = dmin;
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    KM_CUDA(launch_pass_lowd(a, X->prec, X->d, P.nb, ctx->stream));   // partials are sized for P.nb
    return KM_OK;
}

kmeans_status kmeans_energy(kmeans_ctx* ctx, const kmeans_data* X, const void* C, int32_t K, const int32_t* rho,
                            double* E)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, false);
    if (s != KM_OK) return s;
    if (!C || !rho || !E) return fail(ctx, KM_EINVAL, "C, rho and E must not be NULL");
    KM_CUDA(cudaSetDevice(ctx->device));
    const int prec = X->prec == KM_F64 ? KM_F64 : (X->d > 16 ? KM_BF16_F32 : KM_F32);
    Plan P;
    if ((s = make_plan(ctx, X->N, X->d, K, prec, 0, false, P, false)) != KM_OK) return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    if (P.dense) return dense_energy_call(ctx, P, X, C, K, rho, E);
    PassArgs a = base_pass(ctx, P, X->X, X->N, K, prec);
    a.mode = MODE_STANDALONE;
    a.flags = F_ENERGY | (prec != KM_F64 ? F_PACK : 0);
    if (prec == KM_F64) a.c64[0] = reinterpret_cast<const double*>(C);
    else a.rawC = reinterpret_cast<const float*>(C);
    a.rho_in = rho;
    a.out_E = E;
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    KM_CUDA(launch_pass_lowd(a, prec, X->d, P.nb, ctx->stream));   // partials are sized for P.nb
    return KM_OK;
}

kmeans_status kmeans_update(kmeans_ctx* ctx, const kmeans_data* X, const int32_t* rho, int32_t K,
                            const void* C_prev, void* C_out, int64_t* counts)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, false);
    if (s != KM_OK) return s;
    if (!rho || !C_prev || !C_out) return fail(ctx, KM_EINVAL, "rho, C_prev and C_out must not be NULL");
    KM_CUDA(cudaSetDevice(ctx->device));
    const int prec = X->prec == KM_F64 ? KM_F64 : (X->d > 16 ? KM_BF16_F32 : KM_F32);
    Plan P;
    if ((s = make_plan(ctx, X->N, X->d, K, prec, 0, false, P)) != KM_OK) return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    if (P.dense) return dense_update_call(ctx, P, X, rho, K, C_prev, C_out, counts);
    PassArgs a = base_pass(ctx, P, X->X, X->N, K, prec);
    a.mode = MODE_STANDALONE;
    a.flags = F_BINS | (prec != KM_F64 ? F_PACK : 0);
    if (prec == KM_F64) a.c64[0] = reinterpret_cast<const double*>(C_prev);
    else a.rawC = reinterpret_cast<const float*>(C_prev);
    a.rho_in = rho;
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    KM_CUDA(launch_pass_lowd(a, prec, X->d, P.nb, ctx->stream));
    FinArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = MODE_STANDALONE;
    f.K = K;
    f.d = X->d;
    f.nb = P.nb;
    f.part_f64 = prec == KM_F64;
    f.pS = a.pS;
    f.pCnt = a.pCnt;
    f.KB = P.KB;
    f.C_ref = C_prev;
    f.C_out = C_out;
    f.out_f64 = prec == KM_F64;
    f.counts = counts;
    f.st = a.st;
    KM_CUDA(launch_fin(f, P.nfin, ctx->stream));
    return KM_OK;
}

kmeans_status kmeans_solve(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                           const kmeans_params* params, void* C_out, int32_t* rho_out, kmeans_info* info)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, true);
    if (s != KM_OK) return s;
    if (!C0 || !C_out || !rho_out) return fail(ctx, KM_EINVAL, "C0, C_out and rho_out must not be NULL");
    kmeans_params p;
    if (params) p = *params; else kmeans_default_params(&p);
    if ((s = validate_params(ctx, p)) != KM_OK) return s;
    KM_CUDA(cudaSetDevice(ctx->device));
    Plan P;
    if ((s = make_plan(ctx, X->N, X->d, K, X->prec, p.lloyd_only ? 0 : p.m_max, false, P)) != KM_OK) return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    return solve_device(ctx, X, K, C0, p, C_out, rho_out, info, P);
}

kmeans_status kmeans_solve_host(kmeans_ctx* ctx, const kmeans_data* Xh, int32_t K, const void* C0_host,
                                const kmeans_params* params, void* C_out_host, int32_t* rho_out_host,
                                kmeans_info* info)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, Xh, K, true);
    if (s != KM_OK) return s;
    if (!C0_host || !C_out_host || !rho_out_host) return fail(ctx, KM_EINVAL, "NULL host buffer");
    kmeans_params p;
    if (params) p = *params; else kmeans_default_params(&p);
    if ((s = validate_params(ctx, p)) != KM_OK) return s;
    KM_CUDA(cudaSetDevice(ctx->device));
    Plan P;
    if ((s = make_plan(ctx, Xh->N, Xh->d, K, Xh->prec, p.lloyd_only ? 0 : p.m_max, true, P)) != KM_OK) return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    const size_t esz = Xh->prec == KM_F64 ? 8 : 4;
    const size_t n = (size_t)K * Xh->d;
    KM_CUDA(cudaMemcpyAsync(at<void>(ctx, P.hX), Xh->X, (size_t)Xh->N * Xh->d * esz, cudaMemcpyHostToDevice,
                            ctx->stream));
    KM_CUDA(cudaMemcpyAsync(at<void>(ctx, P.hC0), C0_host, n * esz, cudaMemcpyHostToDevice, ctx->stream));
    kmeans_data Xd = *Xh;
    Xd.X = at<void>(ctx, P.hX);
    Xd.X_bf16 = nullptr;
    if (P.dense) {
        KM_CUDA(cudaMemcpyAsync(at<void>(ctx, P.hXb), Xh->X_bf16, (size_t)Xh->N * Xh->d * 2, cudaMemcpyHostToDevice,
                                ctx->stream));
        Xd.X_bf16 = at<void>(ctx, P.hXb);
    }
    s = solve_device(ctx, &Xd, K, at<void>(ctx, P.hC0), p, at<void>(ctx, P.hCout), at<int32_t>(ctx, P.hRho),
                     info, P);
    if (s != KM_OK && s != KM_ENONFINITE) return s;
    KM_CUDA(cudaMemcpyAsync(C_out_host, at<void>(ctx, P.hCout), n * esz, cudaMemcpyDeviceToHost, ctx->stream));
    KM_CUDA(cudaMemcpyAsync(rho_out_host, at<void>(ctx, P.hRho), (size_t)Xh->N * 4, cudaMemcpyDeviceToHost,
                            ctx->stream));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    return s;
}

}  // extern "C"
