// Serving loop (kmeans_server_*): clustering requests of different N, d and K arrive over time.
//
// Admission.  The server owns one device allocation of the stated HBM budget, carved by a
// first-fit allocator (free ranges kept sorted and coalesced).  A request is admitted when its
// device footprint (a copy of X, C0, the results and the solver workspace) fits; low-d requests
// (d <= 16) also need a free batch slot, large requests (d > 16, BF16 distances) a free large
// lane.  Waiting requests are served first come, first served within each class.
//
// Continuous batching.  Low-d requests run in one continuously stepping batch: each
// kmeans_server_step() runs, on the batch stream, the prologue of the requests that joined since
// the last step, one loop pass of Lloyd / Algorithm 1 for every active request (the persistent
// batched kernels of batch.cu over slot-indexed argument tables), and the epilogue and result
// copies of the requests that finished.  Requests join and leave between steps, so a new request
// starts at once instead of waiting for the batch to drain.  Large requests run their whole solve
// graph on the stream of their lane; the GPU overlaps them with the batch steps and each other.
//
// Every request gets bitwise the results of kmeans_solve on it alone: the same kernels with the
// same per-request block decomposition on its own slice of memory.
#include "runtime.cuh"

#include <algorithm>
#include <deque>
#include <map>
#include <vector>

namespace {

// First-fit allocator over [0, cap) in 256-byte granules.
class PoolAlloc {
  public:
    void init(size_t cap)
    {
        free_.clear();
        free_[0] = cap;
        cap_ = cap;
        used_ = 0;
        peak_ = 0;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = al256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = al256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t cap() const { return cap_; }

  private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

enum ReqState { WAITING = 0, JOINING, ACTIVE, FINISHING, COPYING, DONE };

struct Req {
    int64_t ticket = 0;
    kmeans_data Xh{};
    int K = 0;
    const void* C0h = nullptr;
    kmeans_params p{};
    void* Couth = nullptr;
    int32_t* rhoh = nullptr;
    bool large = false;
    int state = WAITING;
    int slot = -1;           // batch slot (low-d) or large lane
    int64_t join_step = 0;
    Plan P{};
    size_t off = 0, bytes = 0;   // pool range (the solver workspace at its start)
    void *Xd = nullptr, *Xbd = nullptr, *C0d = nullptr, *Coutd = nullptr, *infod = nullptr;
    int32_t* rhod = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    kmeans_info info{};
};

constexpr size_t INFO_BYTES = 64;
constexpr size_t SLOT_ITEMS = 8192;   // work items one request may add to a step (all its lists)

}  // namespace

struct kmeans_server {
    kmeans_ctx* ctx = nullptr;
    cudaStream_t s_small = nullptr;
    std::vector<cudaStream_t> s_lane;       // one stream per large lane
    char* pool = nullptr;
    PoolAlloc alloc;
    int S = 0, max_large = 0;
    // device tables, slot-indexed
    char* tab = nullptr;
    size_t t_pass = 0, t_fin = 0, t_mix = 0, t_prep = 0, t_epi = 0, t_st = 0, t_flags = 0, t_items = 0;
    size_t items_cap = 0;
    // pinned host staging
    char* h_tab = nullptr;                  // image of the slot tables
    int* h_flags[2] = {nullptr, nullptr};
    cudaEvent_t ev_flags[2] = {nullptr, nullptr};
    int64_t flags_step[2] = {-1, -1};
    bool flags_open[2] = {false, false};
    int2* h_items[2] = {nullptr, nullptr};
    cudaEvent_t ev_items[2] = {nullptr, nullptr};
    char* h_info = nullptr;                 // [S + max_large] info records
    std::vector<int64_t> slot_req;          // ticket per slot, -1 free
    std::vector<int64_t> lane_req;          // ticket per large lane, -1 free
    std::deque<int64_t> wait_small, wait_large;
    std::map<int64_t, Req> reqs;
    int64_t next_ticket = 1;
    int64_t steps = 0;
    int completed = 0;
    std::string err;
};

namespace {

kmeans_status sfail(kmeans_server* s, kmeans_status st, const std::string& msg)
{
    s->err = msg;
    return st;
}

#define KS_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            char b_[256];                                                          \
            snprintf(b_, sizeof(b_), "%s: %s", #call, cudaGetErrorString(e_));      \
            return sfail(srv, KM_ECUDA, b_);                                       \
        }                                                                          \
    } while (0)

template <typename T>
T* tb(kmeans_server* srv, size_t off)
{
    return reinterpret_cast<T*>(srv->tab + off);
}

size_t esize(const kmeans_data& X) { return X.prec == KM_F64 ? 8 : 4; }

// Upload one slot's entry of table `off` (element size `sz`) from the host image.
cudaError_t put_slot(kmeans_server* srv, size_t off, size_t sz, int slot)
{
    return cudaMemcpyAsync(srv->tab + off + sz * slot, srv->h_tab + off + sz * slot, sz, cudaMemcpyHostToDevice,
                           srv->s_small);
}

// Admission of one low-d request into `slot`: inputs to the device, the slot's tables.
kmeans_status admit_small(kmeans_server* srv, Req& r, int slot)
{
    char* base = srv->pool + r.off;
    const size_t es = esize(r.Xh), n = (size_t)r.K * r.Xh.d;
    KS_CUDA(cudaMemcpyAsync(r.Xd, r.Xh.X, (size_t)r.Xh.N * r.Xh.d * es, cudaMemcpyHostToDevice, srv->s_small));
    KS_CUDA(cudaMemcpyAsync(r.C0d, r.C0h, n * es, cudaMemcpyHostToDevice, srv->s_small));
    kmeans_data Xd = r.Xh;
    Xd.X = r.Xd;
    Xd.X_bf16 = nullptr;
    Xd.X_bf16_lo = nullptr;
    Xd.prec = r.Xh.prec == KM_F64 ? KM_F64 : KM_F32;
    const Launch L = make_launch(base, srv->ctx->nsm, r.P, &Xd, r.K, r.C0d, r.p, r.Coutd, r.rhod);
    PassArgs pa = L.pa;
    pa.nblk = r.P.nb;
    FinArgs fa = L.fa;
    fa.nblk = r.P.nfin;
    const PrepArgs pp = prep_args(L, r.p.m_init);
    const EpiArgs ea = epi_args(L, r.infod);
    SolveState* sp = L.st;
    memcpy(srv->h_tab + srv->t_pass + sizeof(PassArgs) * slot, &pa, sizeof(pa));
    memcpy(srv->h_tab + srv->t_fin + sizeof(FinArgs) * slot, &fa, sizeof(fa));
    memcpy(srv->h_tab + srv->t_mix + sizeof(MixArgs) * slot, &L.ma, sizeof(MixArgs));
    memcpy(srv->h_tab + srv->t_prep + sizeof(PrepArgs) * slot, &pp, sizeof(pp));
    memcpy(srv->h_tab + srv->t_epi + sizeof(EpiArgs) * slot, &ea, sizeof(ea));
    memcpy(srv->h_tab + srv->t_st + sizeof(SolveState*) * slot, &sp, sizeof(sp));
    KS_CUDA(put_slot(srv, srv->t_pass, sizeof(PassArgs), slot));
    KS_CUDA(put_slot(srv, srv->t_fin, sizeof(FinArgs), slot));
    KS_CUDA(put_slot(srv, srv->t_mix, sizeof(MixArgs), slot));
    KS_CUDA(put_slot(srv, srv->t_prep, sizeof(PrepArgs), slot));
    KS_CUDA(put_slot(srv, srv->t_epi, sizeof(EpiArgs), slot));
    KS_CUDA(put_slot(srv, srv->t_st, sizeof(SolveState*), slot));
    r.slot = slot;
    r.state = JOINING;
    r.join_step = srv->steps;
    srv->slot_req[slot] = r.ticket;
    return KM_OK;
}

// A large request runs its whole solve graph on the large stream, then copies its results back.
kmeans_status start_large(kmeans_server* srv, Req& r, int lane)
{
    char* base = srv->pool + r.off;
    const size_t n = (size_t)r.K * r.Xh.d, nx = (size_t)r.Xh.N * r.Xh.d;
    cudaStream_t ls = srv->s_lane[lane];
    KS_CUDA(cudaMemcpyAsync(r.Xd, r.Xh.X, nx * 4, cudaMemcpyHostToDevice, ls));
    KS_CUDA(cudaMemcpyAsync(r.Xbd, r.Xh.X_bf16, nx * 2, cudaMemcpyHostToDevice, ls));
    KS_CUDA(cudaMemcpyAsync(r.C0d, r.C0h, n * 4, cudaMemcpyHostToDevice, ls));
    kmeans_data Xd = r.Xh;
    Xd.X = r.Xd;
    Xd.X_bf16 = r.Xbd;
    Xd.X_bf16_lo = nullptr;         // the prologue splits X on the device
    const Launch L = make_launch(base, srv->ctx->nsm, r.P, &Xd, r.K, r.C0d, r.p, r.Coutd, r.rhod);
    if (!L.maps_ok) return sfail(srv, KM_ECUDA, "cuTensorMapEncodeTiled failed");
    kmeans_status s = record_while_graph(
        srv->ctx, [&](cudaStream_t st) { return launch_prologue(L, st, 0); },
        [&](cudaStream_t st, cudaGraphConditionalHandle h) { return launch_body(L, st, 1, h); },
        [&](cudaStream_t st) { return launch_epilogue(L, st); }, &r.exec);
    if (s != KM_OK) return sfail(srv, s, srv->ctx->err);
    KS_CUDA(cudaGraphLaunch(r.exec, ls));
    char* hinfo = srv->h_info + INFO_BYTES * (size_t)(srv->S + lane);
    KS_CUDA(cudaMemcpyAsync(hinfo, base + r.P.info, devinfo_bytes(), cudaMemcpyDeviceToHost, ls));
    KS_CUDA(cudaMemcpyAsync(r.Couth, r.Coutd, n * 4, cudaMemcpyDeviceToHost, ls));
    KS_CUDA(cudaMemcpyAsync(r.rhoh, r.rhod, (size_t)r.Xh.N * 4, cudaMemcpyDeviceToHost, ls));
    KS_CUDA(cudaEventRecord(r.ev, ls));
    r.slot = lane;
    r.state = COPYING;
    srv->lane_req[lane] = r.ticket;
    return KM_OK;
}

// Footprint and device addresses of a request inside its pool range.
void layout_request(kmeans_server* srv, Req& r)
{
    char* base = srv->pool + r.off;
    const size_t es = r.large ? 4 : esize(r.Xh), n = (size_t)r.K * r.Xh.d, nx = (size_t)r.Xh.N * r.Xh.d;
    size_t o = al256(r.P.total);
    auto take = [&](size_t b) { char* p = base + o; o += al256(b); return p; };
    r.Xd = take(nx * es);
    r.Xbd = r.large ? take(nx * 2) : nullptr;
    r.C0d = take(n * es);
    r.Coutd = take(n * es);
    r.rhod = reinterpret_cast<int32_t*>(take((size_t)r.Xh.N * 4));
    r.infod = take(INFO_BYTES);
}

size_t request_bytes(const Req& r)
{
    const size_t es = r.large ? 4 : esize(r.Xh), n = (size_t)r.K * r.Xh.d, nx = (size_t)r.Xh.N * r.Xh.d;
    return al256(r.P.total) + al256(nx * es) + (r.large ? al256(nx * 2) : 0) + 2 * al256(n * es) +
           al256((size_t)r.Xh.N * 4) + al256(INFO_BYTES);
}

void finish_request(kmeans_server* srv, Req& r, const char* hinfo)
{
    const DevInfoH* di = reinterpret_cast<const DevInfoH*>(hinfo);
    fill_info(&r.info, di, 0.f);
    r.state = DONE;
    srv->alloc.release(r.off, r.bytes);
    if (r.exec) {
        cudaGraphExecDestroy(r.exec);
        r.exec = nullptr;
    }
    if (r.large) srv->lane_req[r.slot] = -1;
    else srv->slot_req[r.slot] = -1;
    srv->completed += 1;
}

// Done flags of step `k` (ring buffer k % 2): active requests that joined at or before step k and
// are done move to FINISHING.
void apply_flags(kmeans_server* srv, int b)
{
    const int64_t k = srv->flags_step[b];
    for (int s = 0; s < srv->S; ++s) {
        if (srv->slot_req[s] < 0 || !srv->h_flags[b][s]) continue;
        Req& r = srv->reqs[srv->slot_req[s]];
        if (r.state == ACTIVE && r.join_step <= k) r.state = FINISHING;
    }
    srv->flags_open[b] = false;
}

struct ItemSet {
    std::vector<std::vector<int2>> pass;   // per group
    std::vector<int2> fin, mix, prep, epi, hp;   // hp: (slot, 0) of the instances passing, for k_hprep
};

struct GroupKey {
    int prec, d, cls;
    size_t smem;
};

kmeans_status server_step(kmeans_server* srv, int32_t* done_now)
{
    const int before = srv->completed;
    // 1. completions (results on the host)
    for (auto& kv : srv->reqs) {
        Req& r = kv.second;
        if (r.state != COPYING) continue;
        const cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) KS_CUDA(q);
        const size_t idx = r.large ? (size_t)(srv->S + r.slot) : (size_t)r.slot;
        finish_request(srv, r, srv->h_info + INFO_BYTES * idx);
    }
    // 2. done flags: at most two steps in flight; apply what has arrived
    const int bcur = (int)(srv->steps & 1);
    if (srv->flags_open[bcur]) {
        KS_CUDA(cudaEventSynchronize(srv->ev_flags[bcur]));
        apply_flags(srv, bcur);
    }
    if (srv->flags_open[bcur ^ 1] && cudaEventQuery(srv->ev_flags[bcur ^ 1]) == cudaSuccess)
        apply_flags(srv, bcur ^ 1);
    // 3. admission
    while (!srv->wait_large.empty()) {
        int lane = -1;
        for (int l = 0; l < srv->max_large; ++l)
            if (srv->lane_req[l] < 0) lane = l;
        if (lane < 0) break;
        Req& r = srv->reqs[srv->wait_large.front()];
        if (!srv->alloc.alloc(r.bytes, &r.off)) break;
        layout_request(srv, r);
        srv->wait_large.pop_front();
        kmeans_status s = start_large(srv, r, lane);
        if (s != KM_OK) return s;
    }
    while (!srv->wait_small.empty()) {
        int slot = -1;
        for (int s = 0; s < srv->S && slot < 0; ++s)
            if (srv->slot_req[s] < 0) slot = s;
        if (slot < 0) break;
        Req& r = srv->reqs[srv->wait_small.front()];
        if (!srv->alloc.alloc(r.bytes, &r.off)) break;
        layout_request(srv, r);
        srv->wait_small.pop_front();
        kmeans_status s = admit_small(srv, r, slot);
        if (s != KM_OK) return s;
    }
    // 4. the batch step
    std::vector<int> J, A, F;
    for (int s = 0; s < srv->S; ++s) {
        if (srv->slot_req[s] < 0) continue;
        const Req& r = srv->reqs[srv->slot_req[s]];
        if (r.state == JOINING) J.push_back(s);
        else if (r.state == ACTIVE) A.push_back(s);
        else if (r.state == FINISHING) F.push_back(s);
    }
    if (J.empty() && A.empty() && F.empty()) {
        *done_now = srv->completed - before;
        return KM_OK;
    }
    std::vector<GroupKey> groups;
    auto group_of = [&](const Req& r) {
        const int prec = r.Xh.prec == KM_F64 ? KM_F64 : KM_F32;
        const int cls = smem_class(r.P.smem);
        for (size_t g = 0; g < groups.size(); ++g)
            if (groups[g].prec == prec && groups[g].d == r.Xh.d && groups[g].cls == cls) {
                groups[g].smem = std::max(groups[g].smem, r.P.smem);
                return (int)g;
            }
        groups.push_back(GroupKey{prec, r.Xh.d, cls, r.P.smem});
        return (int)groups.size() - 1;
    };
    // item lists: prologue (J), body (J + A), epilogue (F)
    ItemSet pro, body, epi;
    size_t fin_smem_max = 0;
    auto add = [&](ItemSet& is, int s, bool pass, bool fin, bool prep, bool epil) {
        const Req& r = srv->reqs[srv->slot_req[s]];
        const int g = group_of(r);
        if ((int)is.pass.size() <= g) is.pass.resize(g + 1);
        if (pass)
            for (int b = 0; b < r.P.nb; ++b) is.pass[g].push_back(make_int2(s, b));
        if (fin) {
            for (int b = 0; b < r.P.nfin; ++b) is.fin.push_back(make_int2(s, b));
            fin_smem_max = std::max(fin_smem_max, fin_smem(r.P.KB, r.Xh.d));
            for (int b = 0; b < mix_blocks(r.K, r.Xh.d); ++b) is.mix.push_back(make_int2(s, b));
        }
        if (prep) is.prep.push_back(make_int2(s, 0));
        if (pass && r.P.ham) is.hp.push_back(make_int2(s, 0));
        if (epil)
            for (int b = 0; b < epi_blocks(r.Xh.N, (size_t)r.K * r.Xh.d); ++b) is.epi.push_back(make_int2(s, b));
    };
    for (int s : J) add(pro, s, true, true, true, false);
    for (int s : J) add(body, s, true, true, false, false);
    for (int s : A) add(body, s, true, true, false, false);
    for (int s : F) add(epi, s, true, false, false, true);
    for (ItemSet* is : {&pro, &body, &epi}) is->pass.resize(groups.size());

    // one upload of every list (pinned staging ring of two)
    std::vector<std::pair<size_t, size_t>> spans;   // (offset in items, count) per list, in order below
    std::vector<const std::vector<int2>*> lists;
    for (ItemSet* is : {&pro, &body, &epi}) {
        for (auto& v : is->pass) lists.push_back(&v);
        lists.push_back(&is->fin);
        lists.push_back(&is->mix);
        lists.push_back(&is->prep);
        lists.push_back(&is->epi);
        lists.push_back(&is->hp);
    }
    size_t tot = 0;
    for (auto* v : lists) {
        spans.emplace_back(tot, v->size());
        tot += v->size();
    }
    if (tot > srv->items_cap) return sfail(srv, KM_ENOMEM, "work-item table full");
    const int ib = (int)(srv->steps & 1);
    KS_CUDA(cudaEventSynchronize(srv->ev_items[ib]));
    for (size_t i = 0; i < lists.size(); ++i)
        if (!lists[i]->empty()) memcpy(srv->h_items[ib] + spans[i].first, lists[i]->data(), sizeof(int2) * lists[i]->size());
    // finished slots leave the done check before this step's kernels run
    for (int s : F) {
        SolveState* nul = nullptr;
        memcpy(srv->h_tab + srv->t_st + sizeof(SolveState*) * s, &nul, sizeof(nul));
        KS_CUDA(put_slot(srv, srv->t_st, sizeof(SolveState*), s));
    }
    if (tot)
        KS_CUDA(cudaMemcpyAsync(srv->tab + srv->t_items, srv->h_items[ib], sizeof(int2) * tot, cudaMemcpyHostToDevice,
                                srv->s_small));
    KS_CUDA(cudaEventRecord(srv->ev_items[ib], srv->s_small));

    int2* items = tb<int2>(srv, srv->t_items);
    const int nsm = srv->ctx->nsm;
    size_t li = 0;
    auto run = [&](ItemSet& is, int mode, int flags, bool with_fin, bool with_prep, bool with_epi) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        const size_t l0 = li;
        li += groups.size() + 5;
        auto hprep = [&](int m) -> cudaError_t {
            if (is.hp.empty()) return cudaSuccess;
            BatchPass h;
            h.args = tb<PassArgs>(srv, srv->t_pass);
            h.items = items + spans[l0 + groups.size() + 4].first;
            h.nitems = (int)is.hp.size();
            h.mode = m;
            h.flags = 0;
            return launch_hprep_batch(h, (int)std::min<size_t>(is.hp.size(), 1024), srv->s_small);
        };
        auto passes = [&](int m) -> cudaError_t {
            cudaError_t r = (m == MODE_INIT || m == MODE_TRIAL) ? hprep(m) : cudaSuccess;
            for (size_t g = 0; g < groups.size() && r == cudaSuccess; ++g) {
                if (is.pass[g].empty()) continue;
                BatchPass b;
                b.args = tb<PassArgs>(srv, srv->t_pass);
                b.items = items + spans[l0 + g].first;
                b.nitems = (int)is.pass[g].size();
                b.mode = m;
                b.flags = flags;
                const int grid = (int)std::min<size_t>(is.pass[g].size(), (size_t)nsm * 2);
                r = launch_pass_lowd_batch(b, groups[g].prec, groups[g].d, grid, groups[g].smem, srv->s_small);
            }
            return r;
        };
        if (with_prep && !is.prep.empty()) {
            BatchPrep p;
            p.args = tb<PrepArgs>(srv, srv->t_prep);
            p.items = items + spans[l0 + groups.size() + 2].first;
            p.nitems = (int)is.prep.size();
            e = launch_prep_batch(p, srv->s_small);
        }
        if (e == cudaSuccess) e = passes(mode);
        if (e == cudaSuccess && mode == MODE_TRIAL) e = passes(MODE_REVERT);
        if (e == cudaSuccess && with_fin && !is.fin.empty()) {
            BatchFin f;
            f.args = tb<FinArgs>(srv, srv->t_fin);
            f.items = items + spans[l0 + groups.size()].first;
            f.nitems = (int)is.fin.size();
            f.mode = mode == MODE_TRIAL ? MODE_TRIAL : MODE_INIT;
            e = launch_fin_batch(f, (int)std::min<size_t>(is.fin.size(), (size_t)nsm * 4), fin_smem_max, srv->s_small);
            if (e == cudaSuccess && !is.mix.empty()) {
                BatchMix m;
                m.args = tb<MixArgs>(srv, srv->t_mix);
                m.items = items + spans[l0 + groups.size() + 1].first;
                m.nitems = (int)is.mix.size();
                m.mode = f.mode;
                e = launch_mix_batch(m, (int)std::min<size_t>(is.mix.size(), (size_t)nsm * 8), srv->s_small);
            }
        }
        if (e == cudaSuccess && with_epi && !is.epi.empty()) {
            BatchEpi ep;
            ep.args = tb<EpiArgs>(srv, srv->t_epi);
            ep.items = items + spans[l0 + groups.size() + 3].first;
            ep.nitems = (int)is.epi.size();
            e = launch_epi_batch(ep, (int)std::min<size_t>(is.epi.size(), (size_t)nsm * 4), srv->s_small);
        }
        return e;
    };
    // Every pass mode runs over all groups (after the bounds' prep) before the next mode starts.
    KS_CUDA(run(pro, MODE_INIT, F_ASSIGN | F_BINS | F_ENERGY | F_CHECK, true, true, false));
    KS_CUDA(run(body, MODE_TRIAL, F_ASSIGN | F_BINS | F_ENERGY | F_CHANGED, true, false, false));
    if (!J.empty() || !A.empty()) {
        BatchDone d;
        d.st = tb<SolveState*>(srv, srv->t_st);
        d.flags = tb<int>(srv, srv->t_flags);
        d.n = srv->S;
        d.loops = reinterpret_cast<unsigned int*>(tb<int>(srv, srv->t_flags) + srv->S);
        d.max_loops = 0xffffffffu;
        d.all_done = tb<int>(srv, srv->t_flags) + srv->S + 1;
        d.use_cond = 0;
        d.cond = 0;
        KS_CUDA(launch_batch_done(d, srv->s_small));
        KS_CUDA(cudaMemcpyAsync(srv->h_flags[bcur], tb<int>(srv, srv->t_flags), sizeof(int) * srv->S,
                                cudaMemcpyDeviceToHost, srv->s_small));
        KS_CUDA(cudaEventRecord(srv->ev_flags[bcur], srv->s_small));
        srv->flags_step[bcur] = srv->steps;
        srv->flags_open[bcur] = true;
    }
    KS_CUDA(run(epi, MODE_EPI, F_ENERGY, false, false, true));
    for (int s : F) {
        Req& r = srv->reqs[srv->slot_req[s]];
        const size_t es = esize(r.Xh);
        KS_CUDA(cudaMemcpyAsync(srv->h_info + INFO_BYTES * (size_t)s, r.infod, devinfo_bytes(), cudaMemcpyDeviceToHost,
                                srv->s_small));
        KS_CUDA(cudaMemcpyAsync(r.Couth, r.Coutd, (size_t)r.K * r.Xh.d * es, cudaMemcpyDeviceToHost, srv->s_small));
        KS_CUDA(cudaMemcpyAsync(r.rhoh, r.rhod, (size_t)r.Xh.N * 4, cudaMemcpyDeviceToHost, srv->s_small));
        KS_CUDA(cudaEventRecord(r.ev, srv->s_small));
        r.state = COPYING;
    }
    for (int s : J) srv->reqs[srv->slot_req[s]].state = ACTIVE;
    srv->steps += 1;
    *done_now = srv->completed - before;
    return KM_OK;
}

}  // namespace

extern "C" {

kmeans_status kmeans_server_create(kmeans_server** out, int device, size_t hbm_budget_bytes, int32_t max_slots,
                                   int32_t max_large)
{
    if (!out || hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 65536 || max_large < 0 || max_large > 64)
        return KM_EINVAL;
    *out = nullptr;
    kmeans_server* srv = new kmeans_server();
    kmeans_status st = kmeans_create(&srv->ctx, device, 0, nullptr);
    if (st != KM_OK) {
        delete srv;
        return st;
    }
    srv->S = max_slots;
    srv->max_large = max_large;
    srv->slot_req.assign((size_t)max_slots, -1);
    srv->lane_req.assign((size_t)std::max(1, max_large), -1);
    srv->items_cap = (size_t)max_slots * SLOT_ITEMS + 65536;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    srv->t_pass = take(sizeof(PassArgs) * max_slots);
    srv->t_fin = take(sizeof(FinArgs) * max_slots);
    srv->t_mix = take(sizeof(MixArgs) * max_slots);
    srv->t_prep = take(sizeof(PrepArgs) * max_slots);
    srv->t_epi = take(sizeof(EpiArgs) * max_slots);
    srv->t_st = take(sizeof(SolveState*) * max_slots);
    srv->t_flags = take(sizeof(int) * (max_slots + 2));
    srv->t_items = take(sizeof(int2) * srv->items_cap);
    const size_t tab_bytes = o;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    ok(cudaStreamCreateWithFlags(&srv->s_small, cudaStreamNonBlocking));
    srv->s_lane.assign((size_t)std::max(1, max_large), nullptr);
    for (auto& ls : srv->s_lane) ok(cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking));
    ok(cudaMalloc(reinterpret_cast<void**>(&srv->tab), tab_bytes));
    if (e == cudaSuccess) ok(cudaMemset(srv->tab, 0, tab_bytes));
    ok(cudaMalloc(reinterpret_cast<void**>(&srv->pool), hbm_budget_bytes));
    ok(cudaHostAlloc(reinterpret_cast<void**>(&srv->h_tab), tab_bytes, cudaHostAllocDefault));
    if (e == cudaSuccess) memset(srv->h_tab, 0, tab_bytes);
    for (int b = 0; b < 2; ++b) {
        ok(cudaHostAlloc(reinterpret_cast<void**>(&srv->h_flags[b]), sizeof(int) * max_slots, cudaHostAllocDefault));
        ok(cudaHostAlloc(reinterpret_cast<void**>(&srv->h_items[b]), sizeof(int2) * srv->items_cap,
                         cudaHostAllocDefault));
        ok(cudaEventCreateWithFlags(&srv->ev_flags[b], cudaEventDisableTiming));
        ok(cudaEventCreateWithFlags(&srv->ev_items[b], cudaEventDisableTiming));
    }
    ok(cudaHostAlloc(reinterpret_cast<void**>(&srv->h_info), INFO_BYTES * (size_t)(max_slots + std::max(1, max_large)),
                     cudaHostAllocDefault));
    if (e == cudaSuccess) ok(cudaEventRecord(srv->ev_items[0], srv->s_small));
    if (e == cudaSuccess) ok(cudaEventRecord(srv->ev_items[1], srv->s_small));
    if (e != cudaSuccess) {
        cudaGetLastError();
        kmeans_server_destroy(srv);
        return e == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA;
    }
    srv->alloc.init(hbm_budget_bytes);
    *out = srv;
    return KM_OK;
}

kmeans_status kmeans_server_destroy(kmeans_server* srv)
{
    if (!srv) return KM_OK;
    if (srv->s_small) cudaStreamSynchronize(srv->s_small);
    for (auto ls : srv->s_lane)
        if (ls) cudaStreamSynchronize(ls);
    for (auto& kv : srv->reqs) {
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    }
    for (int b = 0; b < 2; ++b) {
        if (srv->h_flags[b]) cudaFreeHost(srv->h_flags[b]);
        if (srv->h_items[b]) cudaFreeHost(srv->h_items[b]);
        if (srv->ev_flags[b]) cudaEventDestroy(srv->ev_flags[b]);
        if (srv->ev_items[b]) cudaEventDestroy(srv->ev_items[b]);
    }
    if (srv->h_info) cudaFreeHost(srv->h_info);
    if (srv->h_tab) cudaFreeHost(srv->h_tab);
    if (srv->tab) cudaFree(srv->tab);
    if (srv->pool) cudaFree(srv->pool);
    if (srv->s_small) cudaStreamDestroy(srv->s_small);
    for (auto ls : srv->s_lane)
        if (ls) cudaStreamDestroy(ls);
    kmeans_destroy(srv->ctx);
    delete srv;
    return KM_OK;
}

kmeans_status kmeans_server_submit(kmeans_server* srv, const kmeans_data* Xh, int32_t K, const void* C0_host,
                                   const kmeans_params* params, void* C_out_host, int32_t* rho_out_host,
                                   int64_t* ticket)
{
    if (!srv || !ticket) return KM_EINVAL;
    *ticket = 0;
    kmeans_status s = check_data(srv->ctx, Xh, K, true);
    if (s != KM_OK) return sfail(srv, s, srv->ctx->err);
    if (!C0_host || !C_out_host || !rho_out_host) return sfail(srv, KM_EINVAL, "NULL host buffer");
    Req r;
    if (params) r.p = *params; else kmeans_default_params(&r.p);
    if ((s = validate_params(srv->ctx, r.p)) != KM_OK) return sfail(srv, s, srv->ctx->err);
    r.Xh = *Xh;
    r.K = K;
    r.C0h = C0_host;
    r.Couth = C_out_host;
    r.rhoh = rho_out_host;
    r.large = Xh->d > 16;
    if (r.large && (Xh->prec != KM_BF16_F32 || srv->max_large < 1))
        return sfail(srv, KM_EINVAL, "d > 16 needs KM_BF16_F32 and a large lane");
    if (cudaSetDevice(srv->ctx->device) != cudaSuccess) return sfail(srv, KM_ECUDA, "cudaSetDevice");
    const int prec = r.large ? KM_BF16_F32 : (Xh->prec == KM_F64 ? KM_F64 : KM_F32);
    if ((s = make_plan(srv->ctx, Xh->N, Xh->d, K, prec, r.p.lloyd_only ? 0 : r.p.m_max, false, r.P, true, true)) !=
        KM_OK)
        return sfail(srv, s, srv->ctx->err);
    r.bytes = request_bytes(r);
    if (r.bytes > srv->alloc.cap()) return sfail(srv, KM_ENOMEM, "request larger than the server's HBM budget");
    if (!r.large && 3 * (size_t)r.P.nb + 2 * (size_t)r.P.nfin + 2 * (size_t)mix_blocks(K, Xh->d) + 65 > SLOT_ITEMS)
        return sfail(srv, KM_EINVAL, "request needs more work items than a slot holds");
    if (cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
        return sfail(srv, KM_ECUDA, "cudaEventCreate");
    r.ticket = srv->next_ticket++;
    *ticket = r.ticket;
    (r.large ? srv->wait_large : srv->wait_small).push_back(r.ticket);
    srv->reqs.emplace(r.ticket, r);
    return KM_OK;
}

kmeans_status kmeans_server_step(kmeans_server* srv, int32_t* completed)
{
    if (!srv) return KM_EINVAL;
    int32_t dummy = 0;
    if (cudaSetDevice(srv->ctx->device) != cudaSuccess) return sfail(srv, KM_ECUDA, "cudaSetDevice");
    return server_step(srv, completed ? completed : &dummy);
}

kmeans_status kmeans_server_poll(kmeans_server* srv, int64_t ticket, int32_t* done, kmeans_info* info)
{
    if (!srv || !done) return KM_EINVAL;
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return sfail(srv, KM_EINVAL, "unknown ticket");
    Req& r = it->second;
    *done = r.state == DONE;
    if (!*done) return KM_OK;
    if (info) *info = r.info;
    if (r.ev) cudaEventDestroy(r.ev);
    srv->reqs.erase(it);
    return KM_OK;
}

kmeans_status kmeans_server_get_stats(const kmeans_server* srv, kmeans_server_stats* st)
{
    if (!srv || !st) return KM_EINVAL;
    memset(st, 0, sizeof(*st));
    st->waiting = (int32_t)(srv->wait_small.size() + srv->wait_large.size());
    for (const auto& kv : srv->reqs) {
        const int s = kv.second.state;
        const bool running = s == JOINING || s == ACTIVE || s == FINISHING || s == COPYING;
        if (running && kv.second.large) st->active_large += 1;
        else if (running) st->active_small += 1;
    }
    st->completed = srv->completed;
    st->steps = srv->steps;
    st->pool_bytes = srv->alloc.cap();
    st->pool_used = srv->alloc.used();
    st->pool_peak = srv->alloc.peak();
    return KM_OK;
}

const char* kmeans_server_last_error(const kmeans_server* srv)
{
    return srv ? srv->err.c_str() : "";
}

}  // extern "C"
