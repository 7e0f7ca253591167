// kmeans_update_static: the low-d update step (Eq. 4) with no allocation at all.
//
// Some callers cannot allocate device memory: an allocator or memory pool of their own that calls
// back into K-Means and must not re-enter cudaMalloc, and real-time or embedded programs that
// allocate everything at start-up and treat a later allocation (which synchronises the device) as
// an error.  A context does not suit them either, as its workspace grows on demand.  For them this entry
// point takes no context and keeps its scratch (the per-block partial sums of the pass kernel and
// the last-block counter) in a file-scope __device__ array of fixed size, KM_STATIC_SCRATCH_BYTES.
// Every GPU that loads the library holds that array until the process exits.
//
// The array's host-side name is only a stand-in; its device address is looked up with
// cudaGetSymbolAddress on the first call on a device (with that device current) and cached for
// that device's current CUDA context: a call under a new context (after cudaDeviceReset, or a
// primary context released and made again) looks it up again.  Every call shares the array and
// finds the previous call's contents there: the counter is cleared on each call and the partials
// are fully rewritten.  Calls that overlap on the GPU (different streams, or host threads without
// ordering) race on the array.
//
// The pass uses the block count kmeans_update uses for the same shape (the kernel's occupancy, at
// most 4 blocks per SM, at least 1024 rows per block in FP32 and 256 in FP64), so the two calls sum
// the same partials in the same order and agree bit for bit, unless the array cannot hold that many
// block partials; then fewer blocks are used and FP32 results may differ in the last bits (the
// update stays deterministic for a given device).
#include <mutex>

#include "km_internal.cuh"

namespace km {
namespace {

constexpr size_t KM_STATIC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB
constexpr int KM_STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[KM_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[KM_STATIC_MAX_DEVICES] = {};
void* g_ctx[KM_STATIC_MAX_DEVICES] = {};

// The driver's current context (cuCtxGetCurrent through the runtime's entry-point query, so the
// library needs no link against libcuda); NULL if the query is unavailable.
void* current_context()
{
    typedef int (*CtxGetCurrent)(void**);
    static CtxGetCurrent fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrent>(p);
    }
    void* c = nullptr;
    if (fn && fn(&c) != 0) c = nullptr;
    return c;
}

// Device address of the scratch array on `device` (which must be current), looked up on the first
// call under each context of that device.
cudaError_t scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= KM_STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    void* ctx = current_context();
    if (!g_addr[device] || !ctx || ctx != g_ctx[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);   // makes the device's context current
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
        g_ctx[device] = current_context();
    }
    *out = g_addr[device];
    return cudaSuccess;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace km

using namespace km;

extern "C" kmeans_status kmeans_update_static(const kmeans_data* X, const int32_t* rho, int32_t K,
                                              const void* C_prev, void* C_out, int64_t* counts,
                                              void* cuda_stream)
{
    if (!X || !X->X || !rho || !C_prev || !C_out) return KM_EINVAL;
    if (X->N < 1 || X->d < 1 || X->d > 16 || K < 1 || (int64_t)K > X->N) return KM_EINVAL;
    if (X->prec != KM_F64 && X->prec != KM_F32 && X->prec != KM_BF16_F32) return KM_EINVAL;
    const int d = X->d, prec = X->prec == KM_F64 ? KM_F64 : KM_F32;
    const size_t esz = prec == KM_F64 ? 8 : 4;
    const int Kpad = (K + KPAD_ALIGN - 1) / KPAD_ALIGN * KPAD_ALIGN;
    const size_t smem = pass_lowd_smem(prec, d, K, Kpad, true);
    if (smem > (size_t)LOWD_SMEM_MAX) return KM_EINVAL;   // K*d too large for the per-warp shared-memory bins
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KM_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return KM_ECUDA;
    void* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return KM_ECUDA;

    // partial blocks of the pass: kmeans_update's count for this shape, if the array holds them
    const size_t per_block = al256((size_t)K * d * esz) + al256((size_t)K * 4) + 4 * 64;
    const size_t fixed = 256;
    int per_sm = pass_lowd_occupancy(prec, d, smem);
    per_sm = per_sm > 4 ? 4 : (per_sm < 1 ? 1 : per_sm);
    int64_t nb = (int64_t)nsm * per_sm;
    const int64_t rows = prec == KM_F64 ? LOWD_THREADS : 4 * LOWD_THREADS;
    const int64_t need = (X->N + rows - 1) / rows;
    if (nb > need) nb = need;
    const int64_t fit = (int64_t)((KM_STATIC_SCRATCH_BYTES - fixed) / per_block);
    if (fit < 1) return KM_EINVAL;                 // K*d needs more than KM_STATIC_SCRATCH_BYTES
    if (nb > fit) nb = fit;
    if (nb < 1) nb = 1;

    unsigned char* p = static_cast<unsigned char*>(base);
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* r = p + o; o += al256(bytes); return r; };
    unsigned int* counter = reinterpret_cast<unsigned int*>(take(256));
    void* pS = take((size_t)nb * K * d * esz);
    int32_t* pCnt = reinterpret_cast<int32_t*>(take((size_t)nb * K * 4));
    double* pE = reinterpret_cast<double*>(take((size_t)nb * 8));
    long long* pNch = reinterpret_cast<long long*>(take((size_t)nb * 8));
    long long* pResc = reinterpret_cast<long long*>(take((size_t)nb * 8));
    int* pBad = reinterpret_cast<int*>(take((size_t)nb * 4));
    if (o > KM_STATIC_SCRATCH_BYTES) return KM_EINVAL;

    if (cudaMemsetAsync(counter, 0, 256, s) != cudaSuccess) return KM_ECUDA;
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.X = X->X;
    a.N = X->N;
    a.K = K;
    a.Kpad = Kpad;
    a.mode = MODE_STANDALONE;
    a.flags = F_BINS | (prec != KM_F64 ? F_PACK : 0);
    if (prec == KM_F64)
        a.c64[0] = reinterpret_cast<const double*>(C_prev);
    else
        a.rawC = reinterpret_cast<const float*>(C_prev);
    a.rho_in = rho;
    a.pS = pS;
    a.pCnt = pCnt;
    a.pE = pE;
    a.pNch = pNch;
    a.pResc = pResc;
    a.pBad = pBad;
    a.counter = counter;
    if (launch_pass_lowd(a, prec, d, (int)nb, s) != cudaSuccess) return KM_ECUDA;

    FinArgs f;
    memset(&f, 0, sizeof(f));
    f.mode = MODE_STANDALONE;
    f.K = K;
    f.d = d;
    f.nb = (int)nb;
    f.part_f64 = prec == KM_F64;
    f.pS = pS;
    f.pCnt = pCnt;
    f.C_ref = C_prev;
    f.C_out = C_out;
    f.out_f64 = prec == KM_F64;
    f.counts = counts;
    const int nfin = fin_blocks(K, d, &f.KB);
    if (launch_fin(f, nfin, s) != cudaSuccess) return KM_ECUDA;
    return KM_OK;
}
