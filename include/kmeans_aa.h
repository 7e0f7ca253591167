/*
 * kmeans_aa.h - C ABI of the GB300 (sm_103a) K-Means library with Anderson acceleration.
 *
 * Method: "Fast K-Means Clustering with Anderson Acceleration" (Zhang, Yao, Peng, Yu, Deng).
 * The hot path is one fixed-point step G(C) (Eq. 6) = assignment (Eq. 3) + update (Eq. 4),
 * with the energy E (Eq. 1) fused into the assignment, followed by the Anderson mix
 * (Eq. 7, Eq. 8) under the energy safeguard and the dynamic-m rule of Algorithm 1.
 *
 * Conventions for every call:
 *   - Matrices are row-major.  X is [N, d]; centroids are [K, d].
 *   - Pointers are DEVICE pointers unless the parameter says "host".  The caller owns every
 *     buffer it passes; the library owns only the workspace inside the context.
 *   - Calls are asynchronous on the context's stream, except kmeans_solve and
 *     kmeans_solve_host, which synchronise the stream to fill the host-side info struct.
 *   - Every call returns a kmeans_status; nothing aborts.  kmeans_last_error() gives a
 *     one-line description of the last failure on a context.
 *   - Sizes: 1 <= K <= N (the problem statement of Eq. 1 requires K <= N), 1 <= d <= 4096.
 *     Violations return KM_EINVAL before any work is queued.
 *   - There is no CPU fallback: without a usable GPU every call returns KM_ECUDA.
 */
#ifndef KMEANS_AA_H
#define KMEANS_AA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KM_OK = 0,
    KM_EINVAL = 1,      /* bad argument (shape, NULL pointer, unsupported combination) */
    KM_ENOMEM = 2,      /* workspace would exceed the context's HBM budget, or cudaMalloc failed */
    KM_ECUDA = 3,       /* a CUDA runtime call failed (message in kmeans_last_error) */
    KM_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    KM_ENONFINITE = 5,  /* X or the centroids contain NaN or Inf */
    KM_EBUSY = 6        /* the context is in use by another call */
} kmeans_status;

/* Arithmetic of the distance computation.
 *   KM_F64      X and centroids are double; distances in FP64, direct form sum (x-c)^2.
 *   KM_F32      X and centroids are float; distances as ||c||^2 - 2 x.c in FP32 on CUDA cores
 *               with a per-row error bound; rows whose top-2 gap is inside the bound are
 *               rescored in the direct form in FP32.
 *   KM_BF16_F32 X is float and a BF16 copy of X is supplied (kmeans_data.X_bf16); distances
 *               on tcgen05 tensor cores as BF16 products with FP32 accumulation: X and the
 *               centroids are each split into a BF16 high and low part and the product is the
 *               sum hi.hi + lo.hi + hi.lo (three MMAs), within about 2e-4 |x||c| of the FP32
 *               product; rows whose best two scores lie within that bound are rescored in FP32
 *               from X.  Centroids are float.  Needs 17 <= d <= 128 with d % 8 == 0, K <= 4096,
 *               and X, X_bf16 (and X_bf16_lo if given) 16-byte aligned (else KM_EINVAL).
 *               In the solvers the cluster sums are exact 64-bit integer sums of x * 2^F (F
 *               fixed per solve by max ||x||) carried from pass to pass, so a pass adds only
 *               the rows whose label changed; E follows from them and sum ||x||^2 in FP64.
 * In every mode centroid-space arithmetic (update, residuals, Anderson least squares, energy
 * comparison) is FP64. */
typedef enum { KM_F64 = 0, KM_F32 = 1, KM_BF16_F32 = 2 } kmeans_prec;

/* The samples.  X_bf16 must hold the BF16 rounding of X (to nearest even) when prec ==
 * KM_BF16_F32 and is ignored otherwise.  X_bf16_lo (KM_BF16_F32, optional) holds the BF16 rounding
 * of X - X_bf16, the low part of the split the distance products use; NULL = the library computes it
 * into its workspace (once per solve; on every kmeans_assign call).  The struct itself lives in host
 * memory; X, X_bf16 and X_bf16_lo are device pointers (host pointers for kmeans_solve_host, which
 * always computes the low part on the device). */
typedef struct {
    const void* X;         /* [N, d]: double for KM_F64, float otherwise */
    const void* X_bf16;    /* [N, d] uint16 BF16 bit patterns, KM_BF16_F32 only */
    int64_t N;
    int32_t d;
    int32_t prec;          /* kmeans_prec */
    const void* X_bf16_lo; /* [N, d] uint16 BF16 bit patterns of X - X_bf16, or NULL */
} kmeans_data;

/* Solver parameters (Algorithm 1; defaults from kmeans_default_params):
 *   m_max     maximum history length m-bar (10)
 *   m_init    initial m (2; clamped to m_max)
 *   max_iter  iteration cap (1000)
 *   lloyd_only 1 = plain Lloyd (the same loop with the Anderson step switched off)
 *   eps1, eps2 thresholds of the dynamic-m rule (0.02, 0.5)
 *   tol       0 = stop when the assignment no longer changes (the paper's criterion);
 *             > 0 = stop when at most floor(tol*N) samples change cluster
 *   rank_tol  least-squares columns from the first with |R_kk| <= rank_tol*|R_00| on are dropped
 *             (1e-12), R the triangular factor of the QR of dF (Eq. 7, newest difference first).
 *             The solver reads R off the Cholesky factor of the FP64 Gram matrix while every pivot
 *             ratio exceeds 1e-3 (there the two agree to about 1e-10) and otherwise factors dF by
 *             Householder QR on the device (kmeans_info.ls_qr_solves counts those solves)
 *   fixed_m   1 = keep m at m_init for the whole solve (the fixed-m strategy that Section 3's
 *             "Settings of m" and Tab. 2 compare with the dynamic rule); 0 = dynamic m (default) */
typedef struct {
    int32_t m_max;
    int32_t m_init;
    int32_t max_iter;
    int32_t lloyd_only;
    double eps1;
    double eps2;
    double tol;
    double rank_tol;
    int32_t fixed_m;
} kmeans_params;

/* Result summary (host struct).
 *   iters          loop passes t at termination (Algorithm 1's t; Lloyd counts the same way)
 *   accepted       passes whose accelerated iterate passed the energy safeguard
 *   rejected       passes that reverted to the Lloyd iterate (extra assignment pass each)
 *   assign_passes  assignment passes over X in total (initial + one per t + rejections)
 *   converged      1 = assignment stopped changing, 0 = hit max_iter
 *   m_final        m after the last pass
 *   E              final energy E(P, C) (Eq. 1)
 *   rescored_rows  rows whose reduced-precision top-2 gap was inside the error bound and
 *                  were rescored in FP32, summed over all passes
 *   device_ms      device time of the solve measured with CUDA events (batched solves: of the
 *                  whole batch)
 *   status         kmeans_status of this solve (KM_OK, KM_ENONFINITE, KM_ETIMEOUT)
 *   ls_qr_solves   least-squares solves (Eq. 7) that took the Householder QR route because the
 *                  Cholesky factor of the Gram matrix could not be certified (see kmeans_params)
 *   scanned_rows   rows whose assignment took a scan over all K centroids, summed over the passes
 *                  (the rest were settled by the Hamerly bounds of the FP32 low-d and the
 *                  tensor-core solver passes) */
typedef struct {
    int32_t iters;
    int32_t accepted;
    int32_t rejected;
    int32_t assign_passes;
    int32_t converged;
    int32_t m_final;
    double E;
    int64_t rescored_rows;
    double device_ms;
    int32_t status;
    int32_t ls_qr_solves;
    int64_t scanned_rows;
} kmeans_info;

typedef struct kmeans_ctx kmeans_ctx;

/* Create a context on `device` bound to `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  hbm_budget_bytes caps the workspace the context may allocate
 * (0 = no cap); a call that would exceed it returns KM_ENOMEM.  *ctx is set on success. */
kmeans_status kmeans_create(kmeans_ctx** ctx, int device, size_t hbm_budget_bytes,
                            void* cuda_stream);

/* Free the workspace and the context.  NULL is accepted. */
kmeans_status kmeans_destroy(kmeans_ctx* ctx);

/* Bind a different stream (a cudaStream_t) to the context. */
kmeans_status kmeans_set_stream(kmeans_ctx* ctx, void* cuda_stream);

/* Workspace bytes currently held by the context. */
size_t kmeans_workspace_bytes(const kmeans_ctx* ctx);

/* Static string naming a status code. */
const char* kmeans_status_string(kmeans_status s);

/* Last error message on this context ("" if none).  Valid until the next call. */
const char* kmeans_last_error(const kmeans_ctx* ctx);

/* Fill *p with the defaults listed at kmeans_params. */
void kmeans_default_params(kmeans_params* p);

/* Assignment step, Eq. 3: rho[i] = argmin_j ||x_i - c_j||^2, lowest j on exact ties.
 *   X         samples (see kmeans_data)
 *   C         [K, d] centroids, double for KM_F64 else float
 *   rho       [N] int32 output
 *   rho_prev  [N] int32 previous assignment, or NULL
 *   n_changed device int64 scalar: number of i with rho[i] != rho_prev[i]; requires rho_prev;
 *             may be NULL
 *   dmin      [N] output, X's element type (double or float): the squared distance to the
 *             chosen centroid in the direct form; may be NULL */
kmeans_status kmeans_assign(kmeans_ctx* ctx, const kmeans_data* X, const void* C, int32_t K,
                            int32_t* rho, const int32_t* rho_prev, int64_t* n_changed,
                            void* dmin);

/* Update step, Eq. 4: C_out[j] = mean of the x_i with rho[i] == j; an empty cluster keeps
 * C_prev[j].  Deterministic: the same inputs give bitwise the same output on every run.
 *   rho     [N] int32 in [0, K)
 *   C_prev  [K, d] (element type of X): centroids for empty clusters
 *   C_out   [K, d] output (element type of X); may alias C_prev
 *   counts  [K] int64 output (cluster sizes N_j); may be NULL
 * For d > 16 (FP32 X: the sort-based update of the tensor-core path) X must be 16-byte aligned and
 * d a multiple of 8, d <= 128 (else KM_EINVAL). */
kmeans_status kmeans_update(kmeans_ctx* ctx, const kmeans_data* X, const int32_t* rho,
                            int32_t K, const void* C_prev, void* C_out, int64_t* counts);

/* Energy, Eq. 1, with a given assignment: *E = sum_i ||x_i - c_{rho_i}||^2 (direct form per
 * row in X's precision, accumulated in FP64 in a fixed order).  E is a device double.
 * For d > 16 X must be 16-byte aligned and d a multiple of 8, d <= 128 (else KM_EINVAL). */
kmeans_status kmeans_energy(kmeans_ctx* ctx, const kmeans_data* X, const void* C, int32_t K,
                            const int32_t* rho, double* E);

/* K-Means++ seeding (D^2 sampling; the paper names K-Means++ as an initialiser in Sections 1
 * and 3 without specifying it): C_out[k] = x_{idx[k]}, k = 0..K-1.  idx[0] = floor(u[0] N); then
 * row i is drawn with probability w_i / W, w_i the squared distance from x_i to its nearest row
 * chosen so far (FP64, direct form, separately rounded operations) and W = sum_i w_i, by
 * inverse-CDF sampling in index order with u[k]: the first i whose running sum exceeds u[k] W.
 * If W = 0 (fewer distinct rows than K) idx[k] = floor(u[k] N).
 *   X        [N, d] device (the FP32 copy for KM_BF16_F32; X_bf16 is not used)
 *   u_host   K uniforms in [0, 1), host memory (the caller's random numbers)
 *   C_out    [K, d] device output, element type of X
 *   idx_out  [K] int32 device output, may be NULL
 * Asynchronous on the context's stream; u_host may be reused when the call returns.  Errors:
 * KM_EINVAL (NULL pointers, bad shapes, K > N, N >= 2^31, a u outside [0, 1)), KM_ENOMEM
 * (workspace of 8 N bytes and more past the budget). */
kmeans_status kmeans_seed_pp(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const double* u_host,
                             void* C_out, int32_t* idx_out);

/* Full solve from C0: Lloyd (params->lloyd_only = 1) or Algorithm 1 (Anderson acceleration
 * with the energy safeguard and dynamic m).  All iterations run on the device inside one CUDA
 * graph with a conditional while node; the host only waits for the end.
 *   C0     [K, d] initial centroids (element type of X)
 *   params NULL = defaults
 *   C_out  [K, d] final centroids (element type of X): the means of the final clusters
 *   rho_out [N] int32 final assignment
 *   info   host struct, filled before return (may be NULL) */
kmeans_status kmeans_solve(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                           const kmeans_params* params, void* C_out, int32_t* rho_out,
                           kmeans_info* info);

/* kmeans_solve with HOST buffers: X (and X_bf16), C0, C_out and rho_out are host pointers
 * (pinned memory gives the fastest copies).  The inputs are copied to device workspace, the
 * solve runs, and the results are copied back before return. */
kmeans_status kmeans_solve_host(kmeans_ctx* ctx, const kmeans_data* X_host, int32_t K,
                                const void* C0_host, const kmeans_params* params,
                                void* C_out_host, int32_t* rho_out_host, kmeans_info* info);

/* Anderson least squares, Eq. 7, on the device:  theta = argmin || f - sum_j theta_j dF_j ||^2.
 * The routine of the solver's step, callable on a history the caller supplies.
 *   dF        [m][n] device doubles, difference j+1 contiguous at dF + j n; dF_1 (j = 0) is the
 *             newest difference, the column order the rank rule below refers to
 *   f         [n] device doubles (F^t)
 *   m         1 <= m <= 32 columns;  n >= 1 rows (K*d in the solver)
 *   rank_tol  columns from the first with |R_kk| <= rank_tol |R_00| on are dropped (theta = 0),
 *             R the triangular factor of the QR of dF
 *   method    0 = the solver's rule: the Cholesky factor of the Gram matrix dF^T dF when every
 *             pivot ratio exceeds 1e-3, else Householder QR of [dF | f];  1 = Householder QR
 *             always;  2 = the Gram matrix and its Cholesky factor always (a cross-check: it
 *             squares the condition number)
 *   theta     [m] device double output;  rank, qr_used: device int32 outputs (may be NULL):
 *             columns kept, and 1 if the QR route ran
 * One thread block, asynchronous on the context's stream; uses the context's workspace
 * ((m + 1) n doubles and a small state), so the workspace state of an earlier solve is not kept.
 * KM_EINVAL for NULL pointers or sizes out of range, KM_ENOMEM past the budget. */
kmeans_status kmeans_lsq(kmeans_ctx* ctx, const double* dF, int64_t n, int32_t m, const double* f, double rank_tol,
                         int32_t method, double* theta, int32_t* rank, int32_t* qr_used);

/* The solver's state between two loop passes of Algorithm 1, copied to host memory by
 * kmeans_solve_passes.  The caller supplies the buffers (NULL = not copied); the scalars are filled.
 * After loop pass t (unless the solve ended in it):
 *   C      [K*d] C^{t+1}, the iterate the next pass assigns (the accelerated point, or G^t)
 *   C_AU   [K*d] G^t = Update(P^t) (Algorithm 1's C_AU, the revert target of the next pass)
 *   F      [K*d] F^t = G^t - C^t
 *   dF, dG [m_max][K*d] the differences dF_j = F^{t-j+1} - F^{t-j}, dG_j likewise, newest first
 *          (ring_count of them)
 *   rho    [N] P^t
 *   t      the next pass's t;  m  the current m;  m_t, rank  history length and columns kept by
 *          the last least-squares solve;  theta  its solution (0 past the rank);  from_lloyd 1 if
 *          C is a plain Lloyd iterate;  E_prev, E_prev2  the stored E^t, E^{t-1};  E_trial  E of
 *          the last pass's proposed iterate;  done / converged  the solve ended (then C and rho
 *          hold its result);  accepted, rejected, passes, ls_qr_solves  counters so far.
 * All arithmetic of the state is FP64 whatever the precision of X. */
typedef struct {
    double* C;
    double* C_AU;
    double* F;
    double* dF;
    double* dG;
    int32_t* rho;
    int32_t t, m, m_t, rank, from_lloyd, ring_count, done, converged;
    int32_t accepted, rejected, passes, ls_qr_solves;
    double E_prev, E_prev2, E_trial;
    double theta[32];
} kmeans_state;

/* The solver of kmeans_solve stopped after `passes` loop passes (earlier if it ends), with its
 * state copied to *state: the prologue and each loop pass run the same kernels as kmeans_solve,
 * launched pass by pass from the host.  It exists to check single steps of Algorithm 1 against an
 * independent implementation started from the same state.  C0 and params as for kmeans_solve;
 * passes >= 0.  Synchronous. */
kmeans_status kmeans_solve_passes(kmeans_ctx* ctx, const kmeans_data* X, int32_t K, const void* C0,
                                  const kmeans_params* params, int32_t passes, kmeans_state* state);

/* One instance of a batched solve.  All pointers are device pointers owned by the caller. */
typedef struct {
    kmeans_data X;       /* samples: d <= 16 (KM_F64 or KM_F32), or d > 16 with KM_BF16_F32 and X_bf16 */
    int32_t K;
    const void* C0;      /* [K, d] initial centroids (element type of X) */
    void* C_out;         /* [K, d] final centroids (element type of X) */
    int32_t* rho_out;    /* [N] final assignment */
} kmeans_problem;

/* Solve n independent instances together (Lloyd or Algorithm 1 each, per its parameters).  The
 * low-d instances (d <= 16) advance one loop pass per step; every step of every instance runs
 * inside one CUDA graph launch (a conditional while node that ends when all of them are done),
 * each batched kernel being one persistent grid over (instance, block) work items.  Instances with
 * d > 16 run the tensor-core path as chains of their own in the same graph, beside the low-d chain.
 * Each instance's results are bitwise those of kmeans_solve on it alone (same kernels, same
 * per-instance block decomposition).  The grids of the low-d assignment kernels are picked by
 * timing candidates on the batch's data the first time a batch shape is seen (KM_TUNE=0 in the
 * environment turns that off); the choice does not change any result.
 *   problems  host array of n instances (d > 16 needs KM_BF16_F32 with X_bf16: KM_EINVAL otherwise)
 *   params    host array of n parameter sets, or NULL for the defaults
 *   infos     host array of n results (may be NULL); device_ms is the time of the whole batch
 * Synchronous like kmeans_solve.  Returns the first non-OK instance status (every info is filled). */
kmeans_status kmeans_solve_batched(kmeans_ctx* ctx, const kmeans_problem* problems, int32_t n,
                                   const kmeans_params* params, kmeans_info* infos);

/* One line describing the last batched plan: work-item groups, the timed launch-shape candidates
 * and the grids chosen.  Valid until the next call on the context. */
const char* kmeans_batch_describe(const kmeans_ctx* ctx);

/* ---- Serving: requests of different N, d and K arriving over time ----------------------------
 * A server owns one device allocation of hbm_budget_bytes, carved by a first-fit allocator.  A
 * submitted request waits until its device footprint fits (and, for a low-d request, one of
 * max_slots batch slots is free; for a large request, one of max_large lanes).  Low-d requests
 * (d <= 16) run in one continuously stepping batch: each kmeans_server_step() runs the prologue of
 * newly admitted requests, one loop pass of every active request, and the epilogue and result
 * copies of finished ones, so requests join and leave between steps.  Large requests (d > 16,
 * KM_BF16_F32 with its BF16 copy) run their whole solve on their lane's own stream, overlapping the
 * batch and each other.
 * Each request's results are bitwise those of kmeans_solve on it alone.  A server is used from one
 * host thread. */
typedef struct kmeans_server kmeans_server;

typedef struct {
    int32_t waiting;        /* submitted, not admitted */
    int32_t active_small;   /* admitted low-d requests not yet handed back */
    int32_t active_large;
    int32_t completed;      /* results on the host so far */
    int64_t steps;          /* batch steps run */
    size_t pool_bytes;      /* the HBM budget */
    size_t pool_used;
    size_t pool_peak;
} kmeans_server_stats;

/* Create a server on `device`: 1 <= max_slots <= 65536, 0 <= max_large <= 64.  Allocates the pool
 * (KM_ENOMEM if it does not fit). */
kmeans_status kmeans_server_create(kmeans_server** srv, int device, size_t hbm_budget_bytes, int32_t max_slots,
                                   int32_t max_large);

/* Wait for the server's streams and free everything.  NULL is accepted. */
kmeans_status kmeans_server_destroy(kmeans_server* srv);

/* Queue one request.  X_host, C0_host, C_out_host and rho_out_host are HOST buffers that must stay
 * valid until the request is reported done (pinned memory keeps the copies asynchronous).  The
 * inputs are copied to the device at admission; the results are written to C_out_host and
 * rho_out_host.  *ticket identifies the request.  KM_ENOMEM if the request can never fit. */
kmeans_status kmeans_server_submit(kmeans_server* srv, const kmeans_data* X_host, int32_t K, const void* C0_host,
                                   const kmeans_params* params, void* C_out_host, int32_t* rho_out_host,
                                   int64_t* ticket);

/* Admit what fits, run one batch step, hand back finished requests.  *completed (may be NULL) =
 * requests whose results reached the host during this call.  At most two steps are in flight. */
kmeans_status kmeans_server_step(kmeans_server* srv, int32_t* completed);

/* *done = 1 once the request's results are on the host; info (may be NULL) is then filled and the
 * ticket is released. */
kmeans_status kmeans_server_poll(kmeans_server* srv, int64_t ticket, int32_t* done, kmeans_info* info);

kmeans_status kmeans_server_get_stats(const kmeans_server* srv, kmeans_server_stats* stats);

/* Last error message of the server ("" if none). */
const char* kmeans_server_last_error(const kmeans_server* srv);

/* Measured FP32 FMA throughput of `device` (FMAs per second over all SMs): independent fma.rn.f32
 * chains on 4 blocks of 256 threads per SM, `iters` x 128 FMAs per thread, timed with CUDA events
 * (*ms, may be NULL).  The ALU peak the low-d assignment pass is reported against.  Synchronous;
 * uses the legacy default stream. */
kmeans_status kmeans_measure_fp32_fma(int device, int32_t iters, double* fma_per_s, double* ms);

/* kmeans_update without any allocation, for callers that must not allocate device memory:
 * an allocator or memory pool of the caller's own that calls back into K-Means and must not
 * re-enter cudaMalloc, and real-time or embedded programs that allocate everything at start-up
 * and treat any later allocation (with its device-wide synchronisation) as an error.  Those
 * callers also cannot own a context, whose workspace grows on demand.
 * The paper has no counterpart; it is the same update step (Eq. 4) as kmeans_update.
 *   - No context: the work goes to `cuda_stream` (a cudaStream_t; NULL = legacy default stream)
 *     on the current device.  X, rho, C_prev, C_out and counts are as for kmeans_update.
 *   - Low-d path only: 1 <= d <= 16 (KM_F64, KM_F32; KM_BF16_F32 is treated as KM_F32).
 *   - Scratch: a fixed array of 8 MiB in device memory that the library holds on every GPU that
 *     loads it, until the process exits.  The array stores one block partial of K*d sums and K
 *     counts per thread block.  Shapes are limited first by the pass kernel's shared memory (the
 *     same limit as kmeans_update: K <= 168 in FP64 at d = 16); a shape within that
 *     limit whose single block partial did not fit in 8 MiB would return KM_EINVAL.
 *   - The pass uses kmeans_update's block count for the shape when the array holds that many
 *     block partials (then the two calls agree bit for bit), else as many as it holds (still
 *     deterministic for a given device; FP32 results may then differ from kmeans_update's in the
 *     last bits).
 *   - The first call on a device looks the array's address up (cudaGetSymbolAddress, with that
 *     device current) and caches it for that device's current CUDA context; a call under a new
 *     context (after cudaDeviceReset) looks it up again.  Make the first call on a device before
 *     any stream capture.
 *   - Every call shares the array and leaves its contents behind; each call clears what must
 *     start at zero.  Calls that overlap on the GPU (other streams, unordered host threads) race
 *     on the array: serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Asynchronous on cuda_stream; returns KM_EINVAL for bad arguments, KM_ECUDA if a launch
 *     fails. */
kmeans_status kmeans_update_static(const kmeans_data* X, const int32_t* rho, int32_t K,
                                   const void* C_prev, void* C_out, int64_t* counts,
                                   void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KMEANS_AA_H */
