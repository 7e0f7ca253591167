// Declarations of the dense (tensor-core) assignment and the sort-based update.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "km_internal.cuh"

namespace km {

// TMA descriptors of one dense pass: X's BF16 hi and lo parts ([N][d]) and the centroids' hi and lo
// parts ([Kpad][dpad]) for both centroid sets (0 = C^t, 1 = C_AU).
struct DenseMaps {
    CUtensorMap xh;
    CUtensorMap xl;
    CUtensorMap ch[2];
    CUtensorMap cl[2];
};

// Arguments shared by every kernel of one dense pass (assignment + rescoring + update chain).
struct DenseArgs {
    int64_t N;
    int d;
    int dpad;                 // d rounded up to 64 (BF16 K-blocks of 128 bytes)
    int K;
    int Kpad;                 // K rounded up to 256 (MMA N)
    int mode;                 // PassMode
    const float* X;           // [N][d] FP32
    const __nv_bfloat16* Xb;  // [N][d] BF16 copy x_hi (an MMA operand; its row norms feed the bound)
    const float* cn[2];       // [Kpad] ||c||^2, +inf for pad rows; set 0 = C^t, set 1 = C_AU
    const float* c32[2];      // [K][d] FP32 centroids
    const double* c64[2];     // [K][d] FP64 centroids (C^t, C_AU)
    float bcoef_a;            // error bound B = bcoef_a |x| max|c| + bcoef_b max|c|^2
    float bcoef_b;
    int32_t* rho_out;         // standalone output
    const int32_t* rho_prev;  // standalone previous assignment (optional)
    int32_t* rho_pair[2];     // solver ping-pong assignment
    int* queue;               // [N] near-tie rows to rescore over all K
    void* rkey;               // [N] u64 (distance bits, index) keys of the rescored rows
    unsigned int* qcount;     // [2]: queued rows
    int* err;
    // update chain
    int rows_per_block;
    int* hist;                // [K][nbk] per-block counts -> exclusive scans
    int32_t* counts;          // [K]
    int* off;                 // [K+1] cluster offsets in perm
    int* choff;               // [K] first chunk of each cluster
    int* chunk_cluster;       // [max_chunks]
    int* nchunks;
    int* perm;                // [N]
    float* part;              // [max_chunks][d]
    double* pe;               // [max_chunks / 8]: energy of each k_dsegsum block
    long long* pnch;          // [nbk]
    long long* acc;           // [K][d] int64 fixed-point residual sums (scale 2^counter[3]), read and
    int32_t* accC;            // [K]    cleared by k_fin; cluster sizes
    unsigned int* counter;    // [0]: the update's last block, [1]: k_dscan's, [2]: max |chunk partial|
                              // (FP32 bits), [3]: the pass's fixed-point scale exponent, [4]: max ||x||
                              // (FP32 bits, from k_xcheck), [5]: k_dinc_list's last block, [6]: rows
                              // listed by k_dinc_list, [7]: 1 = this pass rebuilds the sums in full,
                              // [8]: k_xcheck's last block
    int prescaled;            // solver: the scale comes from max ||x|| and max ||c|| before the sums
    // Incremental update of the solver passes (inc != 0).  Spair[i] / Npair[i] hold the exact
    // integer sums of the partition in rho_pair[i]: per cluster the sum of round(x * 2^F) over its
    // rows (F fixed for the solve by max ||x||) and its size.  A pass adds only the rows whose label
    // changed since the last pass (or, past inc_cap such rows and in the INIT pass, rebuilds the sums
    // through the sorted chain); the energy follows from the sums.
    int inc;
    long long inc_cap;
    long long* Spair[2];      // [K][d]
    int32_t* Npair[2];        // [K]
    long long* dS;            // [K][d] this pass's change of the sums (cleared by k_dinc_list)
    int32_t* dN;              // [K]
    double* qx;               // [0]: sum of ||x||^2 over all rows (once per solve); [1..]: k_xcheck's
                              // block partials
    // Hamerly bounds (solver passes; NULL hub: none)
    float* hub;               // [N] upper bound on the distance to the assigned centroid
    float* hlb;               // [N] lower bound on the distance to every other centroid
    const float* xn2;         // [N] ||x||^2 (FP32)
    float* hlast;             // [K][d] the centroids the bounds refer to (the last pass's)
    float* drift;             // [K] drift of each centroid since the last pass
    int* map;                 // [N] rows to scan, compacted (NULL: every row, in order)
    unsigned int* nrows;      // number of rows in map (NULL: N)
    double* out_E;
    long long* out_nch;
    // controller
    SolveState* st;
    long long thr;
    int lloyd_only;
    int fixed_m;
    double eps1;
    double eps2;
    int m_max;
    int max_iter;
    int use_cond;
    cudaGraphConditionalHandle cond;
    int use_cond_rev;                     // TRIAL chain in a graph: sets the REVERT chain's IF node
    cudaGraphConditionalHandle cond_rev;
};

struct PackArgs {
    int K, Kpad, d, dpad, nsets, check_done;
    const double* src64[2];   // FP64 sources (solver) or NULL
    const float* src32;       // FP32 source (standalone)
    __nv_bfloat16* cb[2];     // [Kpad][dpad] hi part
    __nv_bfloat16* cl[2];     // [Kpad][dpad] lo part
    float* cn[2];             // [Kpad]
    float* c32[2];            // [K][d]
    SolveState* st;
};

size_t dense_assign_smem(int dpad, int Kpad);
bool make_tmap_bf16(void* map, const void* base, int64_t rows, int cols, int box_rows);
cudaError_t launch_dense_pass(const DenseArgs& a, const DenseMaps& maps, int nsm, cudaStream_t s);
cudaError_t launch_xsplit(const float* X, const void* Xh, void* Xl, int64_t n, int nsm, cudaStream_t s);
cudaError_t launch_dense_update(const DenseArgs& a, int nbk, int max_chunks, cudaStream_t s);
cudaError_t launch_pack_dense(const PackArgs& p, cudaStream_t s);
cudaError_t launch_drow(const DenseArgs& a, const int32_t* rho_in, float* dmin, double* pe, long long* pn, int blocks,
                        cudaStream_t s);
cudaError_t launch_xcheck(const float* X, int64_t N, int d, unsigned int* xmax, float* xn2, SolveState* st, int nsm,
                          cudaStream_t s, double* qx = nullptr, unsigned int* qctr = nullptr);
// Blocks of k_xcheck (its block partials of sum ||x||^2 need 1 + this many doubles)
int xcheck_blocks(int nsm);
// Hamerly bounds of a solver pass: drifts; then (TRIAL, REVERT) the test per row, the list of rows to
// scan and their BF16 parts copied into the compact buffers Ch, Cl ([N][d] each)
cudaError_t launch_dense_bounds(const DenseArgs& a, const void* Xh, const void* Xl, void* Ch, void* Cl, int nsm,
                                cudaStream_t s);

}  // namespace km
