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
#include "runtime.cuh"

namespace {

kmeans_status record_graph(kmeans_ctx* ctx, const Launch& L)
{
    cudaGraphExec_t exec = nullptr;
    kmeans_status s = record_while_graph(
        ctx, [&](cudaStream_t st) { return launch_prologue(L, st, 0); },
        [&](cudaStream_t st, cudaGraphConditionalHandle h) { return launch_body(L, st, 1, h); },
        [&](cudaStream_t st) { return launch_epilogue(L, st); }, &exec);
    if (s != KM_OK) return s;
    if (ctx->have_graph) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = exec;
    ctx->have_graph = true;
    return KM_OK;
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

kmeans_status solve_device(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                           const kmeans_params& p, void* C_out, int32_t* rho_out, kmeans_info* info,
                           const Plan& P)
{
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.X = X->X;
    key.Xb = X->X_bf16;
    key.Xl = X->X_bf16_lo;
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
    key.ham = P.ham ? 1 + P.hg : 0;
    key.lsq = ls_mode();
    const Launch L = make_launch(arena_base(ctx), ctx->nsm, P, X, K, C0, p, C_out, rho_out);
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
    KM_CUDA(cudaMemcpyAsync(ctx->h_info, at<void>(arena_base(ctx), P.info), sizeof(DevInfoH), cudaMemcpyDeviceToHost,
                            ctx->stream));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    const DevInfoH* di = reinterpret_cast<const DevInfoH*>(ctx->h_info);
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        fill_info(info, di, ms);
    }
    if (di->status == KM_ENONFINITE) return fail(ctx, KM_ENONFINITE, "X contains NaN or Inf");
    if (di->status == KM_ETIMEOUT) return fail(ctx, KM_ETIMEOUT, "iteration guard tripped");
    return KM_OK;
}

// ---- standalone calls on the dense path
kmeans_status dense_pack_user(kmeans_ctx* ctx, const Plan& P, const void* C, int d, int K)
{
    PackArgs pk = pack_args(arena_base(ctx), P, d, K);
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
    DenseArgs a = dense_args(arena_base(ctx), P, X32, X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.Xb = reinterpret_cast<const __nv_bfloat16*>(X->X_bf16);
    a.rho_out = rho;
    a.rho_prev = rho_prev;
    a.out_nch = reinterpret_cast<long long*>(n_changed);
    const void* xlo = dense_xlo(arena_base(ctx), P, X);
    DenseMaps maps;
    if (!dense_maps(arena_base(ctx), P, X->X_bf16, xlo, X->N, X->d, &maps))
        return fail(ctx, KM_ECUDA, "cuTensorMapEncodeTiled failed (X_bf16 and X_bf16_lo must be 16-byte aligned)");
    maps.ch[1] = maps.ch[0];
    maps.cl[1] = maps.cl[0];
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    if (!X->X_bf16_lo)
        KM_CUDA(launch_xsplit(X32, X->X_bf16, const_cast<void*>(xlo), X->N * (int64_t)X->d, ctx->nsm, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_dense_pass(a, maps, ctx->nsm, ctx->stream));
    if (n_changed || dmin)
        KM_CUDA(launch_drow(a, rho, reinterpret_cast<float*>(dmin), at<double>(arena_base(ctx), P.rowe), at<long long>(arena_base(ctx), P.rown),
                            rowred_blocks(ctx), ctx->stream));
    return KM_OK;
}

kmeans_status dense_energy_call(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, const void* C, int K,
                                const int32_t* rho, double* E)
{
    kmeans_status s;
    if ((uintptr_t)X->X & 15u) return fail(ctx, KM_EINVAL, "the energy with d > 16 needs X 16-byte aligned");
    DenseArgs a = dense_args(arena_base(ctx), P, reinterpret_cast<const float*>(X->X), X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.out_E = E;
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_drow(a, rho, nullptr, at<double>(arena_base(ctx), P.rowe), at<long long>(arena_base(ctx), P.rown), rowred_blocks(ctx),
                        ctx->stream));
    return KM_OK;
}

kmeans_status dense_update_call(kmeans_ctx* ctx, const Plan& P, const kmeans_data* X, const int32_t* rho, int K,
                                const void* C_prev, void* C_out, int64_t* counts)
{
    kmeans_status s;
    if ((uintptr_t)X->X & 15u) return fail(ctx, KM_EINVAL, "the update with d > 16 needs X 16-byte aligned");
    DenseArgs a = dense_args(arena_base(ctx), P, reinterpret_cast<const float*>(X->X), X->N, X->d, K);
    a.mode = MODE_STANDALONE;
    a.rho_out = const_cast<int32_t*>(rho);     // read-only here: the labels of the update
    KM_CUDA(cudaMemsetAsync(a.counter, 0, 256, ctx->stream));
    KM_CUDA(cudaMemsetAsync(a.acc, 0, (size_t)K * X->d * 8 + (size_t)K * 4, ctx->stream));
    if ((s = dense_pack_user(ctx, P, C_prev, X->d, K)) != KM_OK) return s;
    KM_CUDA(launch_dense_update(a, P.nbk, P.max_chunks, ctx->stream));
    FinArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = MODE_STANDALONE;
    f.K = K;
    f.d = X->d;
    f.nb = 1;
    f.part_fx = 2;                             // the chain's fixed-point totals
    f.acc = a.acc;
    f.accC = a.accC;
    f.fxs_ptr = reinterpret_cast<const int*>(a.counter + 3);
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
    p->rank_tol = 1e-12;
    p->fixed_m = 0;
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
    if (ctx->have_bgraph) cudaGraphExecDestroy(ctx->bexec);
    if (ctx->h_binfo) cudaFreeHost(ctx->h_binfo);
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
    PassArgs a = base_pass(arena_base(ctx), P, X->X, X->N, K, X->prec);
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
    PassArgs a = base_pass(arena_base(ctx), P, X->X, X->N, K, prec);
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
    PassArgs a = base_pass(arena_base(ctx), P, X->X, X->N, K, prec);
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
    if ((s = make_plan(ctx, X->N, X->d, K, X->prec, p.lloyd_only ? 0 : p.m_max, false, P, true, true, true)) != KM_OK)
        return s;
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
    if ((s = make_plan(ctx, Xh->N, Xh->d, K, Xh->prec, p.lloyd_only ? 0 : p.m_max, true, P, true, true, true)) != KM_OK)
        return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    const size_t esz = Xh->prec == KM_F64 ? 8 : 4;
    const size_t n = (size_t)K * Xh->d;
    KM_CUDA(cudaMemcpyAsync(at<void>(arena_base(ctx), P.hX), Xh->X, (size_t)Xh->N * Xh->d * esz, cudaMemcpyHostToDevice,
                            ctx->stream));
    KM_CUDA(cudaMemcpyAsync(at<void>(arena_base(ctx), P.hC0), C0_host, n * esz, cudaMemcpyHostToDevice, ctx->stream));
    kmeans_data Xd = *Xh;
    Xd.X = at<void>(arena_base(ctx), P.hX);
    Xd.X_bf16 = nullptr;
    Xd.X_bf16_lo = nullptr;         // the prologue splits X on the device
    if (P.dense) {
        KM_CUDA(cudaMemcpyAsync(at<void>(arena_base(ctx), P.hXb), Xh->X_bf16, (size_t)Xh->N * Xh->d * 2, cudaMemcpyHostToDevice,
                                ctx->stream));
        Xd.X_bf16 = at<void>(arena_base(ctx), P.hXb);
    }
    s = solve_device(ctx, &Xd, K, at<void>(arena_base(ctx), P.hC0), p, at<void>(arena_base(ctx), P.hCout), at<int32_t>(arena_base(ctx), P.hRho),
                     info, P);
    if (s != KM_OK && s != KM_ENONFINITE) return s;
    KM_CUDA(cudaMemcpyAsync(C_out_host, at<void>(arena_base(ctx), P.hCout), n * esz, cudaMemcpyDeviceToHost, ctx->stream));
    KM_CUDA(cudaMemcpyAsync(rho_out_host, at<void>(arena_base(ctx), P.hRho), (size_t)Xh->N * 4, cudaMemcpyDeviceToHost,
                            ctx->stream));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    return s;
}

kmeans_status kmeans_lsq(kmeans_ctx* ctx, const double* dF, int64_t n, int32_t m, const double* f, double rank_tol,
                         int32_t method, double* theta, int32_t* rank, int32_t* qr_used)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!dF || !f || !theta) return fail(ctx, KM_EINVAL, "dF, f and theta must not be NULL");
    if (n < 1 || m < 1 || m > MMAX) return fail(ctx, KM_EINVAL, "need n >= 1 and 1 <= m <= 32");
    if (method < 0 || method > 2) return fail(ctx, KM_EINVAL, "method must be 0, 1 or 2");
    if (!(rank_tol >= 0.0)) return fail(ctx, KM_EINVAL, "rank_tol must be >= 0");
    KM_CUDA(cudaSetDevice(ctx->device));
    const size_t st_off = 0, w_off = al256(sizeof(SolveState));
    const size_t total = w_off + al256((size_t)(m + 1) * (size_t)n * 8);
    kmeans_status s = ensure_arena(ctx, total);
    if (s != KM_OK) return s;
    LsqArgs a;
    memset(&a, 0, sizeof(a));
    a.dF = dF;
    a.f = f;
    a.n = (size_t)n;
    a.m = m;
    a.mode = method == 1 ? LS_QR : (method == 2 ? LS_GRAM : LS_AUTO);
    a.rank_tol = rank_tol;
    a.W = at<double>(arena_base(ctx), w_off);
    a.st = at<SolveState>(arena_base(ctx), st_off);
    a.theta = theta;
    a.rank = rank;
    a.qr_used = qr_used;
    KM_CUDA(launch_lsq(a, ctx->stream));
    return KM_OK;
}

kmeans_status kmeans_solve_passes(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                                  const kmeans_params* params, int32_t passes, kmeans_state* state)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kmeans_status s = check_data(ctx, X, K, true);
    if (s != KM_OK) return s;
    if (!C0 || !state) return fail(ctx, KM_EINVAL, "C0 and state must not be NULL");
    if (passes < 0) return fail(ctx, KM_EINVAL, "passes must be >= 0");
    kmeans_params p;
    if (params) p = *params; else kmeans_default_params(&p);
    if ((s = validate_params(ctx, p)) != KM_OK) return s;
    KM_CUDA(cudaSetDevice(ctx->device));
    Plan P;
    if ((s = make_plan(ctx, X->N, X->d, K, X->prec, p.lloyd_only ? 0 : p.m_max, false, P, true, true, true)) != KM_OK)
        return s;
    if ((s = ensure_arena(ctx, P.total)) != KM_OK) return s;
    char* base = arena_base(ctx);
    const Launch L = make_launch(base, ctx->nsm, P, X, K, C0, p, nullptr, nullptr);
    if (!L.maps_ok) return fail(ctx, KM_ECUDA, "cuTensorMapEncodeTiled failed (X_bf16 must be 16-byte aligned)");
    KM_CUDA(launch_prologue(L, ctx->stream, 0));
    for (int i = 0; i < passes; ++i) KM_CUDA(launch_body(L, ctx->stream, 0, 0));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    SolveState hs;
    KM_CUDA(cudaMemcpy(&hs, L.st, sizeof(hs), cudaMemcpyDeviceToHost));
    const size_t n = (size_t)K * X->d;
    if (state->C) KM_CUDA(cudaMemcpy(state->C, at<double>(base, P.C64), n * 8, cudaMemcpyDeviceToHost));
    if (state->C_AU) KM_CUDA(cudaMemcpy(state->C_AU, at<double>(base, P.CAU), n * 8, cudaMemcpyDeviceToHost));
    if (state->F) KM_CUDA(cudaMemcpy(state->F, at<double>(base, P.Fprev), n * 8, cudaMemcpyDeviceToHost));
    const int m_max = L.m_max;
    for (int q = 0; q < hs.ring_count && m_max > 0; ++q) {
        const int slot = (hs.ring_head - q + m_max) % m_max;
        if (state->dF)
            KM_CUDA(cudaMemcpy(state->dF + q * n, at<double>(base, P.dF) + slot * n, n * 8, cudaMemcpyDeviceToHost));
        if (state->dG)
            KM_CUDA(cudaMemcpy(state->dG + q * n, at<double>(base, P.dG) + slot * n, n * 8, cudaMemcpyDeviceToHost));
    }
    // P^t: the buffer the last pass wrote (a pass that did not end the solve flips cur afterwards)
    const int which = hs.done ? hs.cur : (hs.cur ^ 1);
    if (state->rho)
        KM_CUDA(cudaMemcpy(state->rho, which ? L.rhoB : L.rhoA, (size_t)X->N * 4, cudaMemcpyDeviceToHost));
    state->t = hs.t;
    state->m = hs.m;
    state->m_t = hs.m_t;
    state->rank = hs.rank;
    state->from_lloyd = hs.from_lloyd;
    state->ring_count = m_max > 0 ? hs.ring_count : 0;
    state->done = hs.done;
    state->converged = hs.converged;
    state->accepted = hs.accepted;
    state->rejected = hs.rejected;
    state->passes = hs.passes;
    state->ls_qr_solves = hs.ls_qr;
    state->E_prev = hs.E_prev;
    state->E_prev2 = hs.E_prev2;
    state->E_trial = hs.E_trial;
    for (int j = 0; j < 32; ++j) state->theta[j] = j < hs.rank ? hs.theta[j] : 0.0;
    return KM_OK;
}

}  // extern "C"
