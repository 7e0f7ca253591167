/*
 * FP64 CPU oracle for Lloyd's K-Means and Anderson-accelerated K-Means
 * ("Fast K-Means Clustering with Anderson Acceleration", Zhang, Yao, Peng, Yu, Deng).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library and the CUDA
 * library never calls it.
 *
 * Everything is double precision, sequential, in the order the paper states.  The only
 * parallelism is an optional OpenMP loop over samples in the assignment step, where every
 * row is independent and written to its own slot, so results do not depend on the thread
 * count.  Build with -ffp-contract=off so that a*b+c is never fused behind our back.
 *
 * Readings of the paper where it is silent, garbled or self-contradictory are marked with
 * "Reading Rn" and are the same readings the CUDA path implements.
 *
 * Parity pins: every function here is pinned by tests that do not reuse this code
 * (brute force on tiny inputs, library least squares, closed forms, invariants of the
 * method, Anderson acceleration on an affine map, fixed m = 0 against Lloyd, hand-computed
 * inverse-CDF intervals for K-Means++ seeding).  The dynamic-m trajectory on real data
 * is the one part with no external pin (the paper's tables need datasets that are not
 * available); it is checked for the invariants of Algorithm 1 only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------------
 * Assignment step, Eq. 3:  rho_i = argmin_j ||x_i - c_j||.
 * Distances are formed directly as sum_k (x_ik - c_jk)^2 (no norm expansion).  Ties go to
 * the lowest index (Reading R10: the paper does not say; strict '<' in ascending j).
 * dmin_i is the winning squared distance; gap_i = d_(2) - d_(1) (top-2 gap, +inf if K=1).
 * ------------------------------------------------------------------------------------- */
void orc_assign(const double* X, int64_t N, int d, const double* C, int K,
                int32_t* rho, double* dmin, double* gap)
{
    int64_t i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i = 0; i < N; ++i) {
        const double* x = X + i * (int64_t)d;
        double best = INFINITY, second = INFINITY;
        int arg = 0;
        for (int j = 0; j < K; ++j) {
            const double* c = C + (int64_t)j * d;
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
                double t = x[k] - c[k];
                s = s + t * t;
            }
            if (s < best) {
                second = best;
                best = s;
                arg = j;
            } else if (s < second) {
                second = s;
            }
        }
        rho[i] = arg;
        if (dmin) dmin[i] = best;
        if (gap) gap[i] = second - best;
    }
}

/* Energy, Eq. 1, evaluated with a given assignment P:  E(P, C) = sum_i ||x_i - c_{rho_i}||^2,
 * summed sequentially in row order. */
double orc_energy(const double* X, int64_t N, int d, const double* C, const int32_t* rho)
{
    double E = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double* x = X + i * (int64_t)d;
        const double* c = C + (int64_t)rho[i] * d;
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = x[k] - c[k];
            s = s + t * t;
        }
        E = E + s;
    }
    return E;
}

/* Update step, Eq. 4:  c_j = (1/N_j) sum_{rho_i = j} x_i, sums in row order.
 * Reading R9 (the paper divides by N_j and is silent on N_j = 0): an empty cluster keeps
 * its previous centroid C_prev[j]. */
void orc_update(const double* X, int64_t N, int d, const int32_t* rho, int K,
                const double* C_prev, double* C_out, int64_t* counts)
{
    double* S = (double*)calloc((size_t)K * d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) {
        int j = rho[i];
        cnt[j] += 1;
        for (int k = 0; k < d; ++k) S[(int64_t)j * d + k] += X[i * (int64_t)d + k];
    }
    for (int j = 0; j < K; ++j) {
        for (int k = 0; k < d; ++k) {
            int64_t o = (int64_t)j * d + k;
            C_out[o] = cnt[j] > 0 ? S[o] / (double)cnt[j] : C_prev[o];
        }
        if (counts) counts[j] = cnt[j];
    }
    free(S);
    free(cnt);
}

/* ---------------------------------------------------------------------------------------
 * Anderson least-squares problem, Eq. 7:
 *     theta = argmin || f - sum_j theta_j dF_j ||^2
 * dF is n x m, column j stored contiguously at dF + j*n (column 0 = j=1 = newest difference,
 * Reading R2).  Solved by Householder QR of dF without pivoting, applying each reflection to
 * a copy of f.  Reading R11 (the paper only says "an m x m linear system"; it is silent on
 * rank loss): if |R_kk| <= rank_tol * |R_00| (or R_00 = 0), column k and all later (older)
 * columns are dropped and their theta is 0.  Returns the number of columns kept.
 * ------------------------------------------------------------------------------------- */
int orc_ls_qr(const double* dF, int64_t n, int m, const double* f, double rank_tol, double* theta)
{
    for (int j = 0; j < m; ++j) theta[j] = 0.0;
    if (m <= 0 || n <= 0) return 0;
    double* A = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* b = (double*)malloc(sizeof(double) * (size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(A, dF, sizeof(double) * (size_t)n * m);
    memcpy(b, f, sizeof(double) * (size_t)n);
    int steps = m < n ? m : (int)n;
    double R[64];   /* diagonal of R, m <= 64 */
    int rank = 0;
    double r00 = 0.0;
    for (int k = 0; k < steps; ++k) {
        double* a = A + (int64_t)k * n;
        /* norm of a[k:] */
        double nrm = 0.0;
        for (int64_t i = k; i < n; ++i) nrm += a[i] * a[i];
        nrm = sqrt(nrm);
        double alpha = a[k] >= 0.0 ? -nrm : nrm;   /* R_kk = alpha */
        double rkk = fabs(alpha);
        if (k == 0) r00 = rkk;
        if (r00 == 0.0 || rkk <= rank_tol * r00) break;
        /* v = a[k:] - alpha e_k, H = I - 2 v v^T / (v^T v) */
        double vtv = 0.0;
        for (int64_t i = k; i < n; ++i) {
            v[i] = a[i];
            if (i == k) v[i] -= alpha;
            vtv += v[i] * v[i];
        }
        for (int j = k; j < m; ++j) {
            double* aj = A + (int64_t)j * n;
            double s = 0.0;
            for (int64_t i = k; i < n; ++i) s += v[i] * aj[i];
            double w = 2.0 * s / vtv;
            for (int64_t i = k; i < n; ++i) aj[i] -= w * v[i];
        }
        {
            double s = 0.0;
            for (int64_t i = k; i < n; ++i) s += v[i] * b[i];
            double w = 2.0 * s / vtv;
            for (int64_t i = k; i < n; ++i) b[i] -= w * v[i];
        }
        R[k] = A[(int64_t)k * n + k];
        rank = k + 1;
    }
    /* back substitution on the leading rank x rank block: R theta = (Q^T f)[0:rank] */
    for (int k = rank - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < rank; ++j) s -= A[(int64_t)j * n + k] * theta[j];
        theta[k] = s / R[k];
    }
    free(A);
    free(b);
    free(v);
    return rank;
}

/* ---------------------------------------------------------------------------------------
 * Dynamic adjustment of m (Section 2.2, Algorithm 1 "Adjust the value of m"):
 *   ratio = (E^{t-1} - E^t) / (E^{t-2} - E^{t-1});
 *   ratio < eps1 -> m = max(m-1, 0);  ratio > eps2 -> m = min(m+1, m_max).
 * Reading R4: with E^0 = +inf the ratio is undefined or degenerate for t <= 2, so m is only
 * adjusted for t >= 3.  Reading R5: written without the division (num < eps1*den, then
 * num > eps2*den), which is the same test for den > 0 and also covers den = 0.
 * E_cur is E^t of the trial iterate (before any revert); E_prev, E_prev2 are stored energies.
 * ------------------------------------------------------------------------------------- */
int orc_m_rule(int m, int m_max, int t, double E_cur, double E_prev, double E_prev2,
               double eps1, double eps2)
{
    if (t < 3) return m;
    double num = E_prev - E_cur;
    double den = E_prev2 - E_prev;
    if (num < eps1 * den) return m - 1 > 0 ? m - 1 : 0;
    if (num > eps2 * den) return m + 1 < m_max ? m + 1 : m_max;
    return m;
}

/* ---------------------------------------------------------------------------------------
 * Anderson history and accelerated iterate (Eq. 7 and Eq. 8, Algorithm 1 last lines).
 * The history keeps the newest (m_max + 1) pairs (G^s, F^s) in a ring.  aa_mix forms
 *   dF_j = F^{t-j+1} - F^{t-j},  dG_j = G^{t-j+1} - G^{t-j},  j = 1..m_t,
 * solves Eq. 7 and returns C^{t+1} = G^t - sum_j theta_j dG_j.
 * Reading R1: the sign is minus (Algorithm 1; Eq. 8's '+' and 'theta_i' are typos: the
 * minimiser of Eq. 7 makes F^t - dF theta small, whose G-counterpart is G^t - dG theta).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int cap;          /* ring capacity = m_max + 1 */
    int count;        /* number of valid pairs */
    int head;         /* slot of the newest pair */
    int64_t n;        /* vector length (K*d) */
    double* G;        /* cap x n */
    double* F;        /* cap x n */
} orc_hist;

static void hist_init(orc_hist* h, int m_max, int64_t n)
{
    h->cap = m_max + 1;
    h->count = 0;
    h->head = -1;
    h->n = n;
    h->G = (double*)calloc((size_t)h->cap * n, sizeof(double));
    h->F = (double*)calloc((size_t)h->cap * n, sizeof(double));
}

static void hist_free(orc_hist* h)
{
    free(h->G);
    free(h->F);
}

static void hist_push(orc_hist* h, const double* G, const double* F)
{
    h->head = (h->head + 1) % h->cap;
    memcpy(h->G + (int64_t)h->head * h->n, G, sizeof(double) * (size_t)h->n);
    memcpy(h->F + (int64_t)h->head * h->n, F, sizeof(double) * (size_t)h->n);
    if (h->count < h->cap) h->count++;
}

/* pointer to pair s steps back from the newest (s = 0 is the newest) */
static const double* hist_G(const orc_hist* h, int s)
{
    return h->G + (int64_t)((h->head - s + h->cap) % h->cap) * h->n;
}
static const double* hist_F(const orc_hist* h, int s)
{
    return h->F + (int64_t)((h->head - s + h->cap) % h->cap) * h->n;
}

/* Returns the number of LS columns kept (0 means C_next = G^t, a plain Lloyd iterate). */
static int aa_mix(const orc_hist* h, int m_t, double rank_tol, double* C_next, double* theta_out)
{
    int64_t n = h->n;
    const double* Gt = hist_G(h, 0);
    const double* Ft = hist_F(h, 0);
    if (m_t > h->count - 1) m_t = h->count - 1;
    memcpy(C_next, Gt, sizeof(double) * (size_t)n);
    if (m_t <= 0) return 0;
    double* dF = (double*)malloc(sizeof(double) * (size_t)n * m_t);
    double theta[64];
    for (int j = 1; j <= m_t; ++j) {
        const double* Fa = hist_F(h, j - 1);   /* F^{t-j+1} */
        const double* Fb = hist_F(h, j);       /* F^{t-j}   */
        for (int64_t i = 0; i < n; ++i) dF[(int64_t)(j - 1) * n + i] = Fa[i] - Fb[i];
    }
    int rank = orc_ls_qr(dF, n, m_t, Ft, rank_tol, theta);
    for (int j = 1; j <= rank; ++j) {
        const double* Ga = hist_G(h, j - 1);
        const double* Gb = hist_G(h, j);
        for (int64_t i = 0; i < n; ++i) C_next[i] -= theta[j - 1] * (Ga[i] - Gb[i]);
    }
    if (theta_out)
        for (int j = 0; j < m_t; ++j) theta_out[j] = theta[j];
    free(dF);
    return rank;
}

/* ---------------------------------------------------------------------------------------
 * Classical Anderson acceleration (no safeguard, fixed m) on an affine map
 * g(x) = A x + b in R^n, using the same history and mix routine as the K-Means solver.
 * Used by the tests as a textbook pin: for a contraction and m >= n the iterates reach the
 * fixed point (I - A)^{-1} b within about n + 1 steps (Walker & Ni's GMRES equivalence).
 * x holds x^0 on entry and the last iterate on exit.  A is row-major n x n.
 * traj (optional, (iters+1) x n) receives x^0 .. x^iters.
 * ------------------------------------------------------------------------------------- */
void orc_aa_affine(const double* A, const double* b, int n, int m, int iters, double rank_tol,
                   double* x, double* traj)
{
    orc_hist h;
    hist_init(&h, m, n);
    double* g = (double*)malloc(sizeof(double) * n);
    double* f = (double*)malloc(sizeof(double) * n);
    if (traj) memcpy(traj, x, sizeof(double) * n);
    for (int t = 0; t < iters; ++t) {
        for (int r = 0; r < n; ++r) {
            double s = b[r];
            for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
            g[r] = s;
        }
        for (int r = 0; r < n; ++r) f[r] = g[r] - x[r];
        hist_push(&h, g, f);
        int m_t = m < t ? m : t;
        aa_mix(&h, m_t, rank_tol, x, NULL);
        if (traj) memcpy(traj + (int64_t)(t + 1) * n, x, sizeof(double) * n);
    }
    free(g);
    free(f);
    hist_free(&h);
}

/* ---------------------------------------------------------------------------------------
 * Solver: Lloyd (lloyd_only = 1) and Algorithm 1 (Anderson acceleration with dynamic m).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int m_max, m_init, max_iter, lloyd_only;
    double eps1, eps2, tol, rank_tol;
    int fixed_m;         /* 1: m stays at m_init (the fixed-m strategy of Section 3, Tab. 2) */
} orc_params;

typedef struct {
    int iters, accepted, rejected, assign_passes, converged, m_final;
    double E;
} orc_info;

/* one record per pass t = 1..iters of the main loop */
typedef struct {
    int t, n_changed, m, m_t, rank, accelerated, rejected, pad;
    double E_trial;      /* E(P^t, C^t) of the iterate as proposed, before any revert */
    double E;            /* stored E^t */
    double margin_lo;    /* num - eps1*den of the m rule (NaN where the rule is not applied) */
    double margin_hi;    /* num - eps2*den */
    double margin_safe;  /* E_trial - E^{t-1}: the safeguard reverts when this is >= 0 */
} orc_trace;

static int64_t count_changed(const int32_t* a, const int32_t* b, int64_t N)
{
    int64_t c = 0;
    for (int64_t i = 0; i < N; ++i) c += (a[i] != b[i]);
    return c;
}

/*
 * Algorithm 1 with the readings:
 *   R3  the revert target C_AU is G^{t-1}, the Lloyd image of the previous stored iterate;
 *   R4, R5  m rule as in orc_m_rule;
 *   R6  the safeguard reverts on E^t >= E^{t-1} (as written);
 *   R7  after a revert the convergence test is applied again;
 *   R8  convergence is only accepted at a Lloyd iterate: if C^t was an accelerated point and
 *       its assignment equals P^{t-1}, the solver reverts to C_AU (= means of P^{t-1}) and
 *       tests again, so the returned C is always the mean of its clusters;
 *   R13 iters = t at termination; Lloyd runs the same loop, so m_max = 0 reproduces Lloyd;
 *   R14 tol > 0 stops when n_changed <= floor(tol * N); tol = 0 is exact equality;
 *   R18 the safeguard is skipped when C^t is itself a Lloyd iterate (reverting would
 *       re-assign the same point; Lloyd's step never increases E).
 * At max_iter without convergence the returned pair is (P^t, G^t) of the last pass.
 * rho_out (N) and C_out (K*d) are written; trace (optional) gets one record per pass.
 */
int orc_solve(const double* X, int64_t N, int d, int K, const double* C0, const orc_params* p,
              double* C_out, int32_t* rho_out, orc_info* info, orc_trace* trace)
{
    const int64_t n = (int64_t)K * d;
    const int64_t thr = p->tol > 0 ? (int64_t)floor(p->tol * (double)N) : 0;
    const int m_max = p->lloyd_only ? 0 : p->m_max;
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* Pprev = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    double* C = (double*)malloc(sizeof(double) * (size_t)n);
    double* Cnext = (double*)malloc(sizeof(double) * (size_t)n);
    double* CAU = (double*)malloc(sizeof(double) * (size_t)n);
    double* G = (double*)malloc(sizeof(double) * (size_t)n);
    double* F = (double*)malloc(sizeof(double) * (size_t)n);
    orc_hist h;
    hist_init(&h, m_max, n);
    orc_info inf;
    memset(&inf, 0, sizeof(inf));

    /* C^1 = C_AU^1 = G(C^0); F^0 = C^1 - C^0; E^0 = +inf.  P^0 = Assign(C^0). */
    orc_assign(X, N, d, C0, K, Pprev, NULL, NULL);
    inf.assign_passes = 1;
    orc_update(X, N, d, Pprev, K, C0, G, NULL);
    for (int64_t i = 0; i < n; ++i) F[i] = G[i] - C0[i];
    hist_push(&h, G, F);
    memcpy(C, G, sizeof(double) * (size_t)n);
    memcpy(CAU, G, sizeof(double) * (size_t)n);
    int from_lloyd = 1;
    double E_prev = INFINITY, E_prev2 = INFINITY;
    int m = p->m_init < m_max ? p->m_init : m_max;
    if (m < 0) m = 0;
    int done = 0;
    int t;
    for (t = 1; t <= p->max_iter; ++t) {
        orc_trace rec;
        memset(&rec, 0, sizeof(rec));
        rec.t = t;
        rec.accelerated = !from_lloyd;
        rec.margin_lo = rec.margin_hi = NAN;
        /* Check for convergence */
        orc_assign(X, N, d, C, K, P, NULL, NULL);
        inf.assign_passes++;
        int64_t nch = count_changed(P, Pprev, N);
        rec.n_changed = (int)nch;
        int conv = nch <= thr;
        if (conv && from_lloyd) {
            double E = orc_energy(X, N, d, C, P);
            rec.E_trial = rec.E = E;
            rec.margin_safe = NAN;
            rec.m = m;
            if (trace) trace[t - 1] = rec;
            inf.E = E;
            done = 1;
            break;
        }
        /* Adjust the value of m */
        double Et = orc_energy(X, N, d, C, P);
        rec.E_trial = Et;
        if (!p->lloyd_only && !p->fixed_m && t >= 3) {
            double num = E_prev - Et, den = E_prev2 - E_prev;
            rec.margin_lo = num - p->eps1 * den;
            rec.margin_hi = num - p->eps2 * den;
        }
        if (!p->lloyd_only && !p->fixed_m) m = orc_m_rule(m, m_max, t, Et, E_prev, E_prev2, p->eps1, p->eps2);
        rec.m = m;
        rec.margin_safe = Et - E_prev;
        /* Make sure C^t decreases the energy */
        int reject = !from_lloyd && (conv || Et >= E_prev);
        if (reject) {
            memcpy(C, CAU, sizeof(double) * (size_t)n);
            orc_assign(X, N, d, C, K, P, NULL, NULL);
            inf.assign_passes++;
            inf.rejected++;
            rec.rejected = 1;
            Et = orc_energy(X, N, d, C, P);
            nch = count_changed(P, Pprev, N);
            if (nch <= thr) {
                rec.E = Et;
                if (trace) trace[t - 1] = rec;
                inf.E = Et;
                done = 1;
                break;
            }
        } else if (!from_lloyd) {
            inf.accepted++;
        }
        rec.E = Et;
        /* Anderson acceleration */
        orc_update(X, N, d, P, K, C, G, NULL);
        memcpy(CAU, G, sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < n; ++i) F[i] = G[i] - C[i];
        hist_push(&h, G, F);
        int m_t = m < t ? m : t;
        rec.m_t = m_t;
        int rank = 0;
        if (m_t > 0) {
            rank = aa_mix(&h, m_t, p->rank_tol, Cnext, NULL);
        } else {
            memcpy(Cnext, G, sizeof(double) * (size_t)n);
        }
        rec.rank = rank;
        from_lloyd = rank == 0;
        E_prev2 = E_prev;
        E_prev = Et;
        memcpy(Pprev, P, sizeof(int32_t) * (size_t)N);
        memcpy(C, Cnext, sizeof(double) * (size_t)n);
        if (trace) trace[t - 1] = rec;
    }
    if (done) {
        inf.iters = t;
        inf.converged = 1;
        memcpy(C_out, C, sizeof(double) * (size_t)n);
        memcpy(rho_out, P, sizeof(int32_t) * (size_t)N);
    } else {
        inf.iters = p->max_iter;
        inf.converged = 0;
        memcpy(C_out, CAU, sizeof(double) * (size_t)n);
        memcpy(rho_out, Pprev, sizeof(int32_t) * (size_t)N);
        inf.E = orc_energy(X, N, d, CAU, Pprev);
    }
    inf.m_final = m;
    if (info) *info = inf;
    hist_free(&h);
    free(P);
    free(Pprev);
    free(C);
    free(Cnext);
    free(CAU);
    free(G);
    free(F);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * K-Means++ seeding (the D^2 weighting of Arthur and Vassilvitskii, the initialiser the paper
 * names beside random seeding in Sections 1 and 3).  The random numbers are inputs:
 * u[0..K-1], uniform in [0, 1).
 *   i_1 = min(floor(u_0 N), N - 1).
 *   For k >= 2: w_i = min_{j<k} ||x_i - c_j||^2 (direct form), W = sum_i w_i in index order,
 *   S_i = w_0 + ... + w_i; i_k = the smallest i with S_i > u_k W (inverse-CDF sampling), so
 *   sample i is drawn with probability w_i / W and a chosen sample (w = 0) is never drawn again.
 * Reading R22: if W = 0 (fewer than K distinct samples) i_k = min(floor(u_k N), N - 1); if
 *   rounding leaves no S_i above u_k W, the last sample with w_i > 0 is taken.
 * idx (K) gets the chosen rows, C (K*d) their coordinates.
 * ------------------------------------------------------------------------------------- */
void orc_kmeanspp(const double* X, int64_t N, int d, int K, const double* u, int32_t* idx, double* C)
{
    double* w = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t i0 = (int64_t)floor(u[0] * (double)N);
    if (i0 > N - 1) i0 = N - 1;
    if (i0 < 0) i0 = 0;
    idx[0] = (int32_t)i0;
    for (int k = 0; k < d; ++k) C[k] = X[i0 * d + k];
    for (int64_t i = 0; i < N; ++i) w[i] = INFINITY;
    for (int c = 1; c < K; ++c) {
        const double* cp = C + (int64_t)(c - 1) * d;
        double W = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = X[i * d + k] - cp[k];
                s += t * t;
            }
            if (s < w[i]) w[i] = s;
            W += w[i];
        }
        int64_t pick = -1;
        if (W > 0.0) {
            const double target = u[c] * W;
            double S = 0.0;
            int64_t last_pos = -1;
            for (int64_t i = 0; i < N; ++i) {
                if (w[i] > 0.0) last_pos = i;
                S += w[i];
                if (S > target && w[i] > 0.0) {
                    pick = i;
                    break;
                }
            }
            if (pick < 0) pick = last_pos;
        } else {
            pick = (int64_t)floor(u[c] * (double)N);
            if (pick > N - 1) pick = N - 1;
            if (pick < 0) pick = 0;
        }
        idx[c] = (int32_t)pick;
        for (int k = 0; k < d; ++k) C[(int64_t)c * d + k] = X[pick * d + k];
    }
    free(w);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the assignment loop for the calls that follow (results do not depend on it). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
