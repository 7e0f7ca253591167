// Internal declarations shared by the CUDA translation units of libkmeans_aa.
//
// Data layout in HBM (one solve):
//   X [N,d] (caller)            rho ping-pong [2][N] int32      C^t, C_AU, F^{t-1} [K*d] f64
//   dF / dG rings [m_max][K*d] f64 (newest difference at ring_head)
//   packed scoring centroids (FP32 path): [Kpad][DP] f32 = (-2 c'_0 .. -2 c'_{D-1}, ||c'||^2, 0..)
//     with c' = fl32(c - o), o an origin near the data, pad rows (a = 0, ||c'||^2 = +inf)
//   uncentred FP32 centroids [K][D] for the direct-form residual and rescoring
//   per-block partials of one assignment pass: residual sums [nb][K][D], counts [nb][K],
//     energy [nb] f64, changed [nb], rescored [nb]; FP32 solver passes with d <= FX_MAX_D add
//     int64 fixed-point sums into one total [K][D] + counts [K] instead of the per-block sums
//   Hamerly bounds (FP32 low-d solver): upper / lower bound [N] f32 each, the centroids of the
//     last pass [K][D] f32, per-pass drifts / half distances [Kpad] f32 and the drift maxima
//   SolveState: controller scalars, the FP64 Gram matrix of the dF ring, theta.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/kmeans_aa.h"

namespace km {

constexpr int MMAX = 32;            // largest supported m_max (history ring length)
constexpr int KPAD_ALIGN = 16;      // K padded to a multiple of this for the low-d FP32 scan (its chunk widths divide it)
constexpr int LOWD_THREADS = 256;   // threads per block of the low-d pass kernel
constexpr int FIN_THREADS = 256;    // threads per block of the update/finalize kernel
constexpr int DOTS = 2 * MMAX;      // per-block dot partials: Gram row + right-hand side
// FP32 solver passes with d <= FX_MAX_D sum the update in per-block 64-bit fixed point: an exact,
// order-independent add that beats per-warp bins there; with more dimensions the d conversions and
// 64-bit shared-memory adds per sample cost more than the per-warp bins.
constexpr int FX_MAX_D = 4;
// Least squares of Eq. 7 (FinArgs::ls_mode): LS_AUTO solves through the Cholesky factor of the
// incrementally kept Gram matrix when every pivot ratio L_kk / L_00 exceeds LS_CERT_TOL, and by
// Householder QR of dF otherwise; LS_QR always takes the QR; LS_GRAM always the Gram route.  At a
// pivot ratio r the Gram route's R_kk carries a relative error of about u / r^2 (u = 2^-53), so
// above 1e-3 the factor agrees with the QR's R to about 1e-10 and every rank decision at
// rank_tol <= 1e-3 is the QR's.
enum LsMode : int { LS_AUTO = 0, LS_QR = 1, LS_GRAM = 2 };
constexpr double LS_CERT_TOL = 1e-3;
constexpr int LOWD_SMEM_MAX = 227 * 1024;   // opt-in dynamic shared memory per block on sm_103a
constexpr int SM_SMEM = 228 * 1024;         // shared memory per SM

// Pass kinds of the assignment kernel.
enum PassMode : int {
    MODE_STANDALONE = 0,   // kmeans_assign / kmeans_energy / kmeans_update building blocks
    MODE_INIT = 1,         // P^0 = Assign(C^0)
    MODE_TRIAL = 2,        // P^t = Assign(C^t), then the controller (Algorithm 1 head)
    MODE_REVERT = 3,       // only if the controller reverted: P^t = Assign(C_AU)
    MODE_EPI = 4           // after the loop, if it stopped at max_iter: E(P^t, G^t)
};

enum PassFlags : int {
    F_ASSIGN = 1,     // compute rho (else read rho from rho_in)
    F_BINS = 2,       // accumulate per-cluster residual sums and counts
    F_ENERGY = 4,     // accumulate the energy
    F_CHANGED = 8,    // count rho != rho_prev
    F_DMIN = 16,      // write the per-row squared distance
    F_CHECK = 32,     // flag non-finite samples
    F_PACK = 64       // FP32 standalone: pack the raw centroids rawC in every block
};

// Controller and Anderson state of one solve (device resident).
struct SolveState {
    int t;            // current loop pass (Algorithm 1's t), 1-based
    int m;            // current m (dynamic)
    int m_t;          // history length used in the last least-squares solve
    int rank;         // columns kept by the last least-squares solve
    int from_lloyd;   // 1 if C^t is a plain Lloyd iterate (no acceleration)
    int revert;       // 1 if the current pass reverted to C_AU
    int done;
    int converged;
    int accepted;
    int rejected;
    int passes;       // assignment passes so far
    int status;       // kmeans_status of the solve
    int ring_count;   // valid differences in the rings
    int ring_head;    // slot of the newest difference
    int cur;          // which rho buffer holds P^t
    int final_src;    // 0: result is C^t (C64), 1: result is C_AU
    long long n_changed;
    long long rescored;
    long long scanned;    // rows scanned over all K, summed over the assignment passes
    float xmax;           // max |x_ik| over the samples (FP32 path, set by the INIT pass)
    int fx_s;             // scale 2^fx_s of the last pass's fixed-point residual sums (FP32 path)
    int ls_qr;            // least-squares solves that took the Householder QR path
    double E_prev;    // stored E^{t-1}
    double E_prev2;   // stored E^{t-2}
    double E_trial;   // E(P^t, C^t) of the proposed iterate
    double E_cur;     // stored E^t (after any revert)
    double E_final;
    double gram[MMAX * MMAX];
    double bvec[MMAX];
    double theta[MMAX];
    unsigned int ctr_pass;   // last-block counters (reset by the last block)
    unsigned int ctr_fin;
    unsigned int ctr_aux;
    unsigned int body_runs;  // loop body executions (hard iteration guard)
};

// Arguments of the low-d assignment pass (by value).
struct PassArgs {
    const void* X;
    int64_t N;
    int K;
    int Kpad;
    int mode;
    int flags;
    // centroids: [0] = C^t (trial / standalone), [1] = C_AU (revert)
    const float* cpk[2];     // FP32 path packed scoring centroids [Kpad][DP]
    const float* c32[2];     // FP32 path uncentred [K][D]
    const double* c64[2];    // FP64 path [K][D]
    const float* origin;     // FP32 path origin o [D]
    const float* rawC;       // F_PACK: the caller's FP32 centroids [K][D]
    float bound_coef;        // FP32 path: score error bound = bound_coef*max|c'|^2 + bound_coef2*|x'|*max|c'|
    float bound_coef2;
    // assignment buffers: solver uses rho[st->cur] / rho[st->cur ^ 1]
    int32_t* rho[2];
    const int32_t* rho_in;   // standalone: rho to read (no F_ASSIGN) or NULL
    const int32_t* rho_prev; // standalone: previous assignment or NULL
    void* dmin;
    // per-block partials
    void* pS;
    int32_t* pCnt;
    double* pE;
    long long* pNch;
    long long* pResc;
    long long* pScan;        // rows that went through the full scan over K (may be NULL)
    int* pBad;
    unsigned int* counter;
    // FP32 solver passes with fixed-point bins (d <= FX_MAX_D): every block adds its int64 bins and
    // counts into these totals (exact, order-independent) instead of writing block partials.  Zero
    // between uses: the INIT pass clears them, k_fin clears what it read, and a TRIAL pass whose
    // safeguard fired clears them for the REVERT pass.  NULL: block partials as usual.
    long long* acc;          // [K][D]
    int32_t* accC;           // [K]
    // finalize targets
    SolveState* st;
    long long* out_nch;
    double* out_E;
    int use_cond;
    cudaGraphConditionalHandle cond;
    int use_cond_rev;                     // TRIAL pass in a graph: sets the REVERT pass's IF node
    cudaGraphConditionalHandle cond_rev;
    // controller parameters
    int m_max;
    int max_iter;
    int lloyd_only;
    int fixed_m;             // 1 = m stays at its initial value (no dynamic-m rule)
    double eps1;
    double eps2;
    long long thr;
    int nblk;                // blocks of this instance's pass (batched launches only)
    // Hamerly bounds (FP32 solver passes; ham = 0 turns them off): per sample an upper bound on the
    // distance to its assigned centroid and a lower bound on the distance to every other centroid,
    // relative to the centroids of the last pass (hlast, FP32 [K][D])
    int ham;
    int hq_cap;              // rows one block can queue for a full scan (shared memory)
    int d;                   // dimension (the pass kernels also have it as a template argument)
    float* hub;
    float* hlb;
    float* hlast;
    // per-pass inputs of the bounds, written by k_hprep: drift [K], half distance to the nearest
    // other centroid [K], and hm = (largest drift, second largest, index of the largest, eta)
    float* hdr;
    float* hs;
    float* hm;
    // group bounds (hg > 0 groups of centroids, in place of Hamerly's single lower bound and
    // half-distance test): per sample a lower bound on the distance to every centroid of each group
    // other than its own centroid, relative to the centroids of the last pass (hlbg); the groups'
    // largest drift since the last pass (hgd, written by k_hprep with the drifts); the centroids in
    // group order (hperm) and the groups' offsets in it (hgoff), fixed once per solve by k_groups
    int hg;
    float* hlbg;          // [N][hg]
    float* hgd;           // [hg]
    int* hperm;           // [K]
    int* hgoff;           // [hg + 1]
};

// Arguments of the update / Anderson-finalize kernel.
struct FinArgs {
    int mode;             // MODE_STANDALONE (plain update) or MODE_INIT / MODE_TRIAL (solver)
    int K;
    int d;
    int nb;               // number of partial blocks
    int part_f64;         // partial sums are double (else float)
    const void* pS;       // [nb][K][d]
    const int32_t* pCnt;  // [nb][K]
    int KB;               // centroids per block
    int part_fx;          // 1: FP32 low-d solver, TRIAL / REVERT sums are int64 fixed point (scale
                          // st->fx_s); 2: every pass's sums are (dense update chain, scale *fxs_ptr)
    long long* acc;       //   ... accumulated by the pass in acc [K][d] and accC [K] (read, then zeroed)
    int32_t* accC;
    const int* fxs_ptr;   // part_fx == 2: the scale exponent written by the pass
    int inc;              // with part_fx == 2: the sums are the incremental update's raw sums
    const long long* Spair[2];   //   sum of x over each cluster in Spair[st->cur] (scale *fxs_ptr),
    const int32_t* Npair[2];     //   sizes in Npair[st->cur]; kept for the next pass (not zeroed)
    // standalone update
    const void* C_ref;    // reference centroids of the residuals (C_prev), element type T
    void* C_out;          // [K][d] element type T
    int out_f64;
    int64_t* counts;
    // solver
    double* C64;          // C^t
    double* CAU;          // C_AU (in: G^{t-1}, out: G^t)
    double* Fprev;        // F^{t-1} -> F^t
    double* dF;           // [m_max][K*d]
    double* dG;
    double* pDots;        // [gridDim][DOTS]
    SolveState* st;
    int m_max;
    int max_iter;
    int lloyd_only;
    double rank_tol;
    int ls_mode;          // LsMode
    double* qrw;          // [(m_max + 1) * K*d] working matrix of the QR path
    int use_cond;
    cudaGraphConditionalHandle cond;
    // accelerated iterate in the last block (small K*d)
    int fuse_mix;
    int DP;
    int fp32_path;
    const float* origin;
    float* cpk[2];
    float* c32[2];
    int nblk;             // blocks of this instance's finalize launch (batched launches only)
};

// Arguments of the mix + pack kernel.
struct MixArgs {
    int mode;             // MODE_INIT or MODE_TRIAL
    int K;
    int d;
    int Kpad;
    int DP;
    int fp32_path;
    double* C64;
    const double* CAU;
    const double* dG;
    int m_max;
    const float* origin;
    float* cpk[2];
    float* c32[2];
    SolveState* st;
};

// Once-per-solve setup of one instance (k_prep) and its result copy (k_epi).
struct PrepArgs {
    const void* C0;
    int f64;
    int K, d, Kpad, DP, pack;
    double* C64;
    float* origin;
    float* cpk0;
    float* cpk1;
    float* c32_0;
    SolveState* st;
    int m_init, m_max;
    unsigned int* counter;   // the pass counter, cleared here in batched solves
};

struct EpiArgs {
    int f64;
    const SolveState* st;
    const double* C64;
    const double* CAU;
    void* C_out;
    size_t n;
    const int32_t* rhoA;
    const int32_t* rhoB;
    int32_t* rho_out;
    int64_t N;
    void* info;
    int nblk;
};

// kmeans_lsq: Eq. 7 for a caller-supplied history (one block).
struct LsqArgs {
    const double* dF;     // [m][n], column q contiguous, q = 0 the newest difference
    const double* f;      // [n]
    size_t n;
    int m;
    int mode;             // LsMode
    double rank_tol;
    double* W;            // [(m + 1) * n] working matrix of the QR route
    SolveState* st;       // gram / bvec workspace
    double* theta;        // [m] out
    int* rank;            // out, may be NULL
    int* qr_used;         // out, may be NULL
};

// Batched launches: one persistent grid walks a list of work items (instance, block of that
// instance); the per-instance arguments live in device tables.
struct BatchPass {
    const PassArgs* args;
    const int2* items;
    int nitems;
    int mode;
    int flags;
};

struct BatchFin {
    const FinArgs* args;
    const int2* items;
    int nitems;
    int mode;
};

struct BatchMix {
    const MixArgs* args;
    const int2* items;
    int nitems;
    int mode;
};

struct BatchPrep {
    const PrepArgs* args;
    const int2* items;       // (instance, 0)
    int nitems;
};

struct BatchEpi {
    const EpiArgs* args;
    const int2* items;
    int nitems;
};

// End-of-step check of a batched solve: all instances done -> end the graph's while loop.
struct BatchDone {
    SolveState* const* st;   // [n]; NULL entries (free serving slots) are skipped
    int* flags;              // [n] or NULL: st[i]->done per entry, for the host
    int n;
    unsigned int* loops;     // loop passes so far (device counter, cleared by the prologue)
    unsigned int max_loops;  // hard guard: unfinished instances get KM_ETIMEOUT
    int* all_done;           // 1 once every instance is done (read by the host-loop mode)
    int use_cond;
    cudaGraphConditionalHandle cond;
};

// Packed scoring centroids of the FP32 path, pair-interleaved so that one fma.rn.f32x2 scores a
// sample against two centroids: centroids 2p and 2p+1 share a row of 2*DP floats
//   (a_{2p,0}, a_{2p+1,0}, ..., a_{2p,D-1}, a_{2p+1,D-1}, ||c'_{2p}||^2, ||c'_{2p+1}||^2, 0...)
// with a = -2 c'.  Element k of centroid j (k = D is ||c'||^2):
__host__ __device__ inline size_t pk_index(int j, int k, int DP)
{
    return (size_t)(j >> 1) * (2 * DP) + 2 * k + (j & 1);
}

// Host-side launchers (defined in the .cu files).
cudaError_t launch_pass_lowd(const PassArgs& a, int prec, int d, int nb, cudaStream_t s);
size_t pass_lowd_smem(int prec, int d, int K, int Kpad, bool bins, int hq_cap = 0, int hg = 0);
cudaError_t launch_groups(const double* C, int K, int d, int hg, int* perm, int* goff, cudaStream_t s);
int pass_lowd_dp(int d);
cudaError_t launch_fin(const FinArgs& a, int nblocks, cudaStream_t s);
int fin_blocks(int K, int d, int* KB);
cudaError_t launch_mix(const MixArgs& a, cudaStream_t s);
cudaError_t launch_prep(const void* C0, bool f64, int K, int d, int Kpad, int DP, double* C64,
                        float* origin, float* cpk0, float* cpk1, float* c32_0, SolveState* st, int m_init,
                        int m_max, cudaStream_t s, int pack = 1);
cudaError_t launch_epi(bool f64, const SolveState* st, const double* C64, const double* CAU, void* C_out,
                       size_t n, const int32_t* rhoA, const int32_t* rhoB, int32_t* rho_out, int64_t N,
                       void* info, cudaStream_t s);
size_t devinfo_bytes();
cudaError_t launch_lsq(const LsqArgs& a, cudaStream_t s);

// Batched launchers (persistent grids over work items).
// variant: 0 = the default rows per thread of the scan, 1 = half of them (FP32 only; same results)
cudaError_t launch_pass_lowd_batch(const BatchPass& b, int prec, int d, int grid, size_t smem, cudaStream_t s,
                                   int variant = 0);
int pass_lowd_batch_occupancy(int prec, int d, size_t smem, int variant = 0);
constexpr int LOWD_BATCH_VARIANTS = 2;
int pass_lowd_occupancy(int prec, int d, size_t smem);   // resident blocks per SM (CUDA occupancy API)
int pass_lowd_occupancy_ao(int d, size_t smem);          // the same for the FP32 assignment-only kernel
cudaError_t launch_hprep(const PassArgs& a, int mode, cudaStream_t s);
cudaError_t launch_hprep_batch(const BatchPass& b, int grid, cudaStream_t s);
cudaError_t launch_fin_batch(const BatchFin& b, int grid, size_t smem, cudaStream_t s);
size_t fin_smem(int KB, int d);
cudaError_t launch_mix_batch(const BatchMix& b, int grid, cudaStream_t s);
cudaError_t launch_prep_batch(const BatchPrep& b, cudaStream_t s);
cudaError_t launch_epi_batch(const BatchEpi& b, int grid, cudaStream_t s);
cudaError_t launch_batch_done(const BatchDone& b, cudaStream_t s);

}  // namespace km
