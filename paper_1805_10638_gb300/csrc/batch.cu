// Batched solves (kmeans_solve_batched): many independent instances of different N, d and K
// advance together, one loop pass of Lloyd or Algorithm 1 per step, all steps inside one CUDA
// graph with a conditional while node:
//
//   prologue : k_prep_batch -> pass(INIT) per (precision, d) group -> k_fin_batch(INIT)
//              -> k_mix_batch(INIT)
//   while    : pass(TRIAL) per group -> pass(REVERT) per group -> k_fin_batch -> k_mix_batch
//              -> k_batch_done (ends the loop once every instance is done)
//   epilogue : pass(EPI) per group -> k_epi_batch
//
// Every batched kernel is a persistent grid over work items (instance, block of that instance).
// An item does what that block of the instance's own launch does, on the instance's own slice of
// the workspace and with the instance's own block count, so each instance gets bitwise the
// results of kmeans_solve on it alone.  The grid sizes (launch shapes) change only the speed; an
// autotuner picks the pass kernels' grids by timing candidates on the batch's own data.
//
// Instances with d > 16 (tensor-core path, BF16 distances) join the same graph as chains of their
// own (their standalone prologue / while / epilogue), independent of the low-d chain, so one
// launch runs the whole batch and the GPU overlaps the chains.
#include "runtime.cuh"

#include <algorithm>
#include <vector>

namespace {

constexpr size_t INFO_STRIDE = 64;

struct BInst {
    Plan P;
    size_t off;
    int group;
    int nepi;
    bool dense;
};

struct BGroup {
    int prec;        // KM_F64 or KM_F32
    int d;
    int cls;         // shared-memory class (smem_class)
    double ops;      // sum of N*K*(d+2) over its instances (ALU work of one pass, for reports)
    size_t smem;
    std::vector<int2> items;
    size_t items_off;
    int grid;
    int variant;     // launch shape of the pass kernel: 0 = default rows per thread, 1 = half (FP32)
};

struct BLayout {
    size_t tables;   // first table byte (after the instance slices)
    size_t t_pass, t_tune, t_fin, t_mix, t_prep, t_epi, t_st, t_info, t_prep_items, t_fin_items, t_mix_items,
        t_epi_items, t_ctl;
    size_t total;
};

struct Batch {
    int n = 0;
    int n_lowd = 0;
    bool any_ham = false;
    std::vector<Launch> dense;       // d > 16 instances: their own solve chains in the same graph
    std::vector<BInst> inst;
    std::vector<BGroup> groups;
    std::vector<int2> fin_items, mix_items, epi_items;
    size_t fin_smem_max = 0;
    int grid_fin = 1, grid_mix = 1, grid_epi = 1;
    unsigned int max_loops = 0;
    BLayout L{};
    char* base = nullptr;
};

template <typename T>
T* bat(const Batch& B, size_t off)
{
    return reinterpret_cast<T*>(B.base + off);
}

BatchPass pass_launch(const Batch& B, const BGroup& g, int mode, int flags, bool tune)
{
    BatchPass b;
    b.args = bat<PassArgs>(B, tune ? B.L.t_tune : B.L.t_pass);
    b.items = bat<int2>(B, g.items_off);
    b.nitems = (int)g.items.size();
    b.mode = mode;
    b.flags = flags;
    return b;
}

cudaError_t batch_passes(const Batch& B, int mode, int flags, cudaStream_t s)
{
    if (B.any_ham && (mode == MODE_INIT || mode == MODE_TRIAL)) {   // REVERT: from the TRIAL pass
        BatchPass h;
        h.args = bat<PassArgs>(B, B.L.t_pass);
        h.items = bat<int2>(B, B.L.t_prep_items);
        h.nitems = B.n_lowd;
        h.mode = mode;
        h.flags = 0;
        cudaError_t e = launch_hprep_batch(h, std::min(B.n_lowd, 1024), s);
        if (e != cudaSuccess) return e;
    }
    for (const BGroup& g : B.groups) {
        cudaError_t e =
            launch_pass_lowd_batch(pass_launch(B, g, mode, flags, false), g.prec, g.d, g.grid, g.smem, s, g.variant);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_fin(const Batch& B, int mode, cudaStream_t s)
{
    BatchFin f;
    f.args = bat<FinArgs>(B, B.L.t_fin);
    f.items = bat<int2>(B, B.L.t_fin_items);
    f.nitems = (int)B.fin_items.size();
    f.mode = mode;
    cudaError_t e = launch_fin_batch(f, B.grid_fin, B.fin_smem_max, s);
    if (e != cudaSuccess || B.mix_items.empty()) return e;
    BatchMix m;
    m.args = bat<MixArgs>(B, B.L.t_mix);
    m.items = bat<int2>(B, B.L.t_mix_items);
    m.nitems = (int)B.mix_items.size();
    m.mode = mode;
    return launch_mix_batch(m, B.grid_mix, s);
}

BatchDone done_args(const Batch& B, int use_cond, cudaGraphConditionalHandle h)
{
    BatchDone d;
    d.st = bat<SolveState*>(B, B.L.t_st);
    d.flags = nullptr;
    d.n = B.n;
    d.loops = bat<unsigned int>(B, B.L.t_ctl);
    d.max_loops = B.max_loops;
    d.all_done = bat<int>(B, B.L.t_ctl + 4);
    d.use_cond = use_cond;
    d.cond = h;
    return d;
}

cudaError_t batch_prologue(const Batch& B, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(B.base + B.L.t_ctl, 0, 256, s);
    BatchPrep p;
    p.args = bat<PrepArgs>(B, B.L.t_prep);
    p.items = bat<int2>(B, B.L.t_prep_items);
    p.nitems = B.n_lowd;
    if (e == cudaSuccess) e = launch_prep_batch(p, s);
    if (e == cudaSuccess) e = batch_passes(B, MODE_INIT, F_ASSIGN | F_BINS | F_ENERGY | F_CHECK, s);
    if (e == cudaSuccess) e = batch_fin(B, MODE_INIT, s);
    return e;
}

cudaError_t batch_body(const Batch& B, cudaStream_t s, int use_cond, cudaGraphConditionalHandle h)
{
    const int fl = F_ASSIGN | F_BINS | F_ENERGY | F_CHANGED;
    cudaError_t e = batch_passes(B, MODE_TRIAL, fl, s);
    if (e == cudaSuccess) e = batch_passes(B, MODE_REVERT, fl, s);
    if (e == cudaSuccess) e = batch_fin(B, MODE_TRIAL, s);
    if (e == cudaSuccess) e = launch_batch_done(done_args(B, use_cond, h), s);
    return e;
}

cudaError_t batch_epilogue(const Batch& B, cudaStream_t s)
{
    cudaError_t e = batch_passes(B, MODE_EPI, F_ENERGY, s);
    BatchEpi ep;
    ep.args = bat<EpiArgs>(B, B.L.t_epi);
    ep.items = bat<int2>(B, B.L.t_epi_items);
    ep.nitems = (int)B.epi_items.size();
    if (e == cudaSuccess) e = launch_epi_batch(ep, B.grid_epi, s);
    return e;
}

// Launch shapes of the pass kernels, per group of instances (precision, d, shared-memory class),
// picked by timing on the batch's own data.  After running the batch's prologue (so every instance
// holds its packed C^1), time for each group a pass that does the loop pass's work (assignment,
// bins, energy) for every candidate: the kernel variant (FP32: the default rows per thread of the
// scan or half of them, which trades registers and instruction-level parallelism against
// occupancy) x the persistent grid (1 block per SM up to the variant's occupancy limit, and one
// block per work item); keep the fastest.  Every candidate gives bitwise the same results (same
// rows per block, same order of the per-thread sums), so the choice only changes the speed.  The
// timed passes write only scratch (the second assignment buffer and the block partials); the
// solve's own prologue runs again afterwards.
kmeans_status tune_batch(kmeans_ctx* ctx, Batch& B, std::string& desc)
{
    const char* env = getenv("KM_TUNE");
    const bool tune = !(env && env[0] == '0') && B.n_lowd > 0;
    char buf[256];
    for (BGroup& g : B.groups) {
        const char* fv = getenv("KM_BATCH_VARIANT");
        g.variant = fv && g.prec != KM_F64 ? std::min(std::max(atoi(fv), 0), LOWD_BATCH_VARIANTS - 1) : 0;
        const int occ = pass_lowd_batch_occupancy(g.prec, g.d, g.smem, g.variant);
        g.grid = std::min((int)g.items.size(), ctx->nsm * std::min(occ, 2));
    }
    if (tune) KM_CUDA(batch_prologue(B, ctx->stream));
    for (size_t gi = 0; gi < B.groups.size(); ++gi) {
        BGroup& g = B.groups[gi];
        const int nit = (int)g.items.size();
        const int nvar = g.prec == KM_F64 ? 1 : LOWD_BATCH_VARIANTS;
        const char* fv = getenv("KM_BATCH_VARIANT");     // restrict the tuner to one variant (tests)
        const int v0 = fv && nvar > 1 ? std::min(std::max(atoi(fv), 0), nvar - 1) : 0;
        const int v1 = fv && nvar > 1 ? v0 + 1 : nvar;
        snprintf(buf, sizeof(buf), "%s d=%d cls=%d ops=%.6g items=%d", g.prec == KM_F64 ? "f64" : "f32", g.d, g.cls,
                 g.ops, nit);
        desc += buf;
        if (tune) {
            const BatchPass b = pass_launch(B, g, MODE_STANDALONE, F_ASSIGN | F_BINS | F_ENERGY, true);
            float best = 1e30f;
            for (int v = v0; v < v1; ++v) {
                const int occ = pass_lowd_batch_occupancy(g.prec, g.d, g.smem, v);
                std::vector<int> cand;
                for (int bps = 1; bps <= occ; ++bps) cand.push_back(std::min(nit, ctx->nsm * bps));
                cand.push_back(nit);
                std::sort(cand.begin(), cand.end());
                cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
                snprintf(buf, sizeof(buf), " v%d(occ %d)", v, occ);
                desc += buf;
                for (int grid : cand) {
                    KM_CUDA(launch_pass_lowd_batch(b, g.prec, g.d, grid, g.smem, ctx->stream, v));
                    KM_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
                    for (int r = 0; r < 3; ++r) KM_CUDA(launch_pass_lowd_batch(b, g.prec, g.d, grid, g.smem, ctx->stream, v));
                    KM_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
                    KM_CUDA(cudaEventSynchronize(ctx->ev1));
                    float ms = 0.f;
                    KM_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
                    ms /= 3.f;
                    snprintf(buf, sizeof(buf), " %d:%.1fus", grid, ms * 1e3f);
                    desc += buf;
                    if (ms < best) {
                        best = ms;
                        g.grid = grid;
                        g.variant = v;
                    }
                }
            }
        }
        snprintf(buf, sizeof(buf), " -> variant %d grid %d; ", g.variant, g.grid);
        desc += buf;
    }
    return KM_OK;
}

// Serialised identity of a batch: the problems, parameters and workspace it was recorded for.
std::string batch_key(const kmeans_problem* pr, int n, const std::vector<kmeans_params>& ps, const kmeans_ctx* ctx)
{
    std::string k;
    k.append(reinterpret_cast<const char*>(&n), sizeof(n));
    k.append(reinterpret_cast<const char*>(pr), sizeof(kmeans_problem) * (size_t)n);
    k.append(reinterpret_cast<const char*>(ps.data()), sizeof(kmeans_params) * (size_t)n);
    k.append(reinterpret_cast<const char*>(&ctx->arena), sizeof(ctx->arena));
    k.append(reinterpret_cast<const char*>(&ctx->arena_bytes), sizeof(ctx->arena_bytes));
    k.push_back(hamerly_mode() ? 'H' : 'h');
    return k;
}

kmeans_status batch_solve(kmeans_ctx* ctx, const kmeans_problem* pr, int n, const kmeans_params* params,
                          kmeans_info* infos)
{
    std::vector<kmeans_params> ps((size_t)n);
    kmeans_status s;
    for (int i = 0; i < n; ++i) {
        if (params) ps[i] = params[i]; else kmeans_default_params(&ps[i]);
        if ((s = validate_params(ctx, ps[i])) != KM_OK) return s;
        const kmeans_problem& q = pr[i];
        if ((s = check_data(ctx, &q.X, q.K, false)) != KM_OK) return s;
        if (!q.C0 || !q.C_out || !q.rho_out) return fail(ctx, KM_EINVAL, "C0, C_out and rho_out must not be NULL");
        if (q.X.d > 16 && (q.X.prec != KM_BF16_F32 || !q.X.X_bf16))
            return fail(ctx, KM_EINVAL, "batched instances with d > 16 need KM_BF16_F32 and X_bf16");
    }
    Batch B;
    B.n = n;
    B.inst.resize((size_t)n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        const kmeans_problem& q = pr[i];
        BInst& bi = B.inst[i];
        bi.dense = q.X.d > 16;
        const int prec = bi.dense ? KM_BF16_F32 : (q.X.prec == KM_F64 ? KM_F64 : KM_F32);
        if ((s = make_plan(ctx, q.X.N, q.X.d, q.K, prec, ps[i].lloyd_only ? 0 : ps[i].m_max, false, bi.P, true,
                           true)) != KM_OK)
            return s;
        bi.off = o;
        o += al256(bi.P.total);
        bi.group = -1;
        bi.nepi = 0;
        if (bi.dense) continue;
        B.n_lowd += 1;
        B.any_ham = B.any_ham || bi.P.ham;
        int gi = -1;
        for (size_t g = 0; g < B.groups.size(); ++g)
            if (B.groups[g].prec == prec && B.groups[g].d == q.X.d && B.groups[g].cls == smem_class(bi.P.smem))
                gi = (int)g;
        if (gi < 0) {
            BGroup g;
            g.prec = prec;
            g.d = q.X.d;
            g.cls = smem_class(bi.P.smem);
            g.ops = 0.0;
            g.smem = 0;
            g.items_off = 0;
            g.grid = 1;
            g.variant = 0;
            B.groups.push_back(g);
            gi = (int)B.groups.size() - 1;
        }
        bi.group = gi;
        BGroup& g = B.groups[gi];
        g.smem = std::max(g.smem, bi.P.smem);
        g.ops += (double)q.X.N * q.K * (q.X.d + 2);
        for (int b = 0; b < bi.P.nb; ++b) g.items.push_back(make_int2(i, b));
        for (int b = 0; b < bi.P.nfin; ++b) B.fin_items.push_back(make_int2(i, b));
        B.fin_smem_max = std::max(B.fin_smem_max, fin_smem(bi.P.KB, q.X.d));
        for (int b = 0; b < mix_blocks(q.K, q.X.d); ++b) B.mix_items.push_back(make_int2(i, b));
        bi.nepi = epi_blocks(q.X.N, (size_t)q.K * q.X.d);
        for (int b = 0; b < bi.nepi; ++b) B.epi_items.push_back(make_int2(i, b));
        B.max_loops = std::max(B.max_loops, (unsigned int)ps[i].max_iter + 3u);
    }
    // device tables after the instance slices
    BLayout& L = B.L;
    L.tables = o;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    L.t_pass = take(sizeof(PassArgs) * (size_t)n);
    L.t_tune = take(sizeof(PassArgs) * (size_t)n);
    L.t_fin = take(sizeof(FinArgs) * (size_t)n);
    L.t_mix = take(sizeof(MixArgs) * (size_t)n);
    L.t_prep = take(sizeof(PrepArgs) * (size_t)n);
    L.t_epi = take(sizeof(EpiArgs) * (size_t)n);
    L.t_st = take(sizeof(SolveState*) * (size_t)n);
    L.t_info = take(INFO_STRIDE * (size_t)n);
    for (BGroup& g : B.groups) g.items_off = take(sizeof(int2) * g.items.size());
    L.t_prep_items = take(sizeof(int2) * (size_t)n);
    L.t_fin_items = take(sizeof(int2) * std::max<size_t>(1, B.fin_items.size()));
    L.t_mix_items = take(sizeof(int2) * std::max<size_t>(1, B.mix_items.size()));
    L.t_epi_items = take(sizeof(int2) * std::max<size_t>(1, B.epi_items.size()));
    L.t_ctl = take(256);
    L.total = o;
    if ((s = ensure_arena(ctx, L.total)) != KM_OK) return s;
    if (devinfo_bytes() > INFO_STRIDE) return fail(ctx, KM_EINVAL, "internal: info record too large");
    B.base = arena_base(ctx);

    // host image of the tables
    std::vector<unsigned char> img(L.total - L.tables, 0);
    auto put = [&](size_t off, const void* src, size_t bytes) { memcpy(img.data() + (off - L.tables), src, bytes); };
    for (int i = 0; i < n; ++i) {
        const kmeans_problem& q = pr[i];
        BInst& bi = B.inst[i];
        char* ib = B.base + bi.off;
        Launch Ln = make_launch(ib, ctx->nsm, bi.P, &q.X, q.K, q.C0, ps[i], q.C_out, q.rho_out);
        if (bi.dense) {
            if (!Ln.maps_ok) return fail(ctx, KM_ECUDA, "cuTensorMapEncodeTiled failed (X_bf16 must be 16-byte aligned)");
            Ln.info = B.base + L.t_info + (size_t)i * INFO_STRIDE;
            B.dense.push_back(Ln);
            continue;
        }
        PassArgs pa = Ln.pa;
        pa.nblk = bi.P.nb;
        put(L.t_pass + i * sizeof(PassArgs), &pa, sizeof(pa));
        PassArgs tu = pa;          // standalone mode on the packed C^1 the prologue leaves
        tu.rho[0] = Ln.rhoB;
        put(L.t_tune + i * sizeof(PassArgs), &tu, sizeof(tu));
        FinArgs fa = Ln.fa;
        fa.nblk = bi.P.nfin;
        put(L.t_fin + i * sizeof(FinArgs), &fa, sizeof(fa));
        put(L.t_mix + i * sizeof(MixArgs), &Ln.ma, sizeof(MixArgs));
        const PrepArgs pp = prep_args(Ln, ps[i].m_init);
        put(L.t_prep + i * sizeof(PrepArgs), &pp, sizeof(pp));
        const EpiArgs ea = epi_args(Ln, B.base + L.t_info + (size_t)i * INFO_STRIDE);
        put(L.t_epi + i * sizeof(EpiArgs), &ea, sizeof(ea));
        SolveState* sp = Ln.st;
        put(L.t_st + i * sizeof(SolveState*), &sp, sizeof(sp));
    }
    for (const BGroup& g : B.groups) put(g.items_off, g.items.data(), sizeof(int2) * g.items.size());
    {
        std::vector<int2> pi;
        for (int i = 0; i < n; ++i)
            if (!B.inst[i].dense) pi.push_back(make_int2(i, 0));
        if (!pi.empty()) put(L.t_prep_items, pi.data(), sizeof(int2) * pi.size());
    }
    if (!B.fin_items.empty()) put(L.t_fin_items, B.fin_items.data(), sizeof(int2) * B.fin_items.size());
    if (!B.mix_items.empty()) put(L.t_mix_items, B.mix_items.data(), sizeof(int2) * B.mix_items.size());
    if (!B.epi_items.empty()) put(L.t_epi_items, B.epi_items.data(), sizeof(int2) * B.epi_items.size());
    KM_CUDA(cudaMemcpyAsync(B.base + L.tables, img.data(), img.size(), cudaMemcpyHostToDevice, ctx->stream));

    B.grid_fin = (int)std::max<size_t>(1, std::min<size_t>(B.fin_items.size(), (size_t)ctx->nsm * 4));
    B.grid_mix = (int)std::max<size_t>(1, std::min<size_t>(B.mix_items.size(), (size_t)ctx->nsm * 8));
    B.grid_epi = (int)std::max<size_t>(1, std::min<size_t>(B.epi_items.size(), (size_t)ctx->nsm * 4));

    const std::string key = batch_key(pr, n, ps, ctx);
    const bool use_graph = graph_mode();
    if (!ctx->have_bgraph || key != ctx->bkey) {
        std::string desc;
        if ((s = tune_batch(ctx, B, desc)) != KM_OK) return s;
        char buf[128];
        snprintf(buf, sizeof(buf), "fin items=%zu grid=%d; mix items=%zu; epi items=%zu; tensor-core chains=%zu",
                 B.fin_items.size(), B.grid_fin, B.mix_items.size(), B.epi_items.size(), B.dense.size());
        desc += buf;
        if (ctx->have_bgraph) {
            cudaGraphExecDestroy(ctx->bexec);
            ctx->have_bgraph = false;
        }
        cudaGraphExec_t exec = nullptr;
        if (use_graph) {
            // one graph: the low-d chain and one chain per tensor-core instance, all independent
            cudaGraph_t g = nullptr;
            KM_CUDA(cudaGraphCreate(&g, 0));
            if (B.n_lowd > 0)
                s = add_while_chain(
                    ctx, g, [&](cudaStream_t st) { return batch_prologue(B, st); },
                    [&](cudaStream_t st, cudaGraphConditionalHandle h) { return batch_body(B, st, 1, h); },
                    [&](cudaStream_t st) { return batch_epilogue(B, st); });
            for (size_t k = 0; k < B.dense.size() && s == KM_OK; ++k) {
                const Launch& Ld = B.dense[k];
                s = add_while_chain(
                    ctx, g, [&](cudaStream_t st) { return launch_prologue(Ld, st, 0); },
                    [&](cudaStream_t st, cudaGraphConditionalHandle h) { return launch_body(Ld, st, 1, h); },
                    [&](cudaStream_t st) { return launch_epilogue(Ld, st); });
            }
            if (s == KM_OK) {
                const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
                if (e != cudaSuccess) s = cuda_fail(ctx, e, "cudaGraphInstantiate");
            }
            cudaGraphDestroy(g);
            if (s != KM_OK) return s;
        }
        ctx->bexec = exec;
        ctx->have_bgraph = use_graph;
        ctx->bkey = use_graph ? key : std::string();
        ctx->bdesc = desc;
        ctx->bgrids.clear();
        for (const BGroup& g : B.groups) ctx->bgrids.push_back(g.grid);
    } else {
        for (size_t g = 0; g < B.groups.size(); ++g) B.groups[g].grid = ctx->bgrids[g];
    }

    KM_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
    if (use_graph) {
        KM_CUDA(cudaGraphLaunch(ctx->bexec, ctx->stream));
    } else {
        int* done = reinterpret_cast<int*>(static_cast<char*>(ctx->h_info) + 128);
        if (B.n_lowd > 0) {
            KM_CUDA(batch_prologue(B, ctx->stream));
            for (unsigned int it = 0; it <= B.max_loops; ++it) {
                KM_CUDA(batch_body(B, ctx->stream, 0, 0));
                KM_CUDA(cudaMemcpyAsync(done, B.base + L.t_ctl + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
                KM_CUDA(cudaStreamSynchronize(ctx->stream));
                if (*done) break;
            }
            KM_CUDA(batch_epilogue(B, ctx->stream));
        }
        for (const Launch& Ld : B.dense) {
            KM_CUDA(launch_prologue(Ld, ctx->stream, 0));
            for (int it = 0; it < Ld.p.max_iter + 2; ++it) {
                KM_CUDA(launch_body(Ld, ctx->stream, 0, 0));
                KM_CUDA(cudaMemcpyAsync(done, &Ld.st->done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
                KM_CUDA(cudaStreamSynchronize(ctx->stream));
                if (*done) break;
            }
            KM_CUDA(launch_epilogue(Ld, ctx->stream));
        }
    }
    KM_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
    const size_t ib = INFO_STRIDE * (size_t)n;
    if (ctx->h_binfo_bytes < ib) {
        if (ctx->h_binfo) cudaFreeHost(ctx->h_binfo);
        ctx->h_binfo = nullptr;
        ctx->h_binfo_bytes = 0;
        KM_CUDA(cudaHostAlloc(&ctx->h_binfo, ib, cudaHostAllocDefault));
        ctx->h_binfo_bytes = ib;
    }
    KM_CUDA(cudaMemcpyAsync(ctx->h_binfo, B.base + L.t_info, ib, cudaMemcpyDeviceToHost, ctx->stream));
    KM_CUDA(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    kmeans_status first = KM_OK;
    for (int i = 0; i < n; ++i) {
        const DevInfoH* di =
            reinterpret_cast<const DevInfoH*>(static_cast<const char*>(ctx->h_binfo) + (size_t)i * INFO_STRIDE);
        if (infos) fill_info(&infos[i], di, ms);
        if (first == KM_OK && di->status != KM_OK) first = (kmeans_status)di->status;
    }
    if (first == KM_ENONFINITE) return fail(ctx, first, "an instance's X contains NaN or Inf");
    if (first == KM_ETIMEOUT) return fail(ctx, first, "iteration guard tripped in an instance");
    return first;
}

}  // namespace

extern "C" {

kmeans_status kmeans_solve_batched(kmeans_ctx* ctx, const kmeans_problem* problems, int32_t n,
                                   const kmeans_params* params, kmeans_info* infos)
{
    if (!ctx) return KM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!problems || n < 1) return fail(ctx, KM_EINVAL, "need n >= 1 problems");
    KM_CUDA(cudaSetDevice(ctx->device));
    return batch_solve(ctx, problems, n, params, infos);
}

const char* kmeans_batch_describe(const kmeans_ctx* ctx)
{
    return ctx ? ctx->bdesc.c_str() : "";
}

}  // extern "C"
