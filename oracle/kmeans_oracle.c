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
 * The history holds the differences
 *   dF_j = F^{t-j+1} - F^{t-j},  dG_j = G^{t-j+1} - G^{t-j},  j = 1..count  (count <= m_max),
 * newest first: dF_1 at dF[0].  Each new pair (G^t, F^t) pushes dF_1 = F^t - F^{t-1} and
 * dG_1 = G^t - G^{t-1} in front and drops the oldest difference once m_max are kept.
 * aa_mix solves Eq. 7 over the newest m_t differences and returns C^{t+1} = G^t - sum_j theta_j dG_j.
 * Reading R1: the sign is minus (Algorithm 1; Eq. 8's '+' and 'theta_i' are typos: the
 * minimiser of Eq. 7 makes F^t - dF theta small, whose G-counterpart is G^t - dG theta).
 * ------------------------------------------------------------------------------------- */
static void hist_push(double* dF, double* dG, int* count, int m_max, int64_t n, const double* G_new,
                      const double* G_old, const double* F_new, const double* F_old)
{
    if (m_max <= 0) return;
    int keep = *count < m_max ? *count : m_max - 1;
    memmove(dF + n, dF, sizeof(double) * (size_t)n * keep);
    memmove(dG + n, dG, sizeof(double) * (size_t)n * keep);
    for (int64_t i = 0; i < n; ++i) {
        dF[i] = F_new[i] - F_old[i];
        dG[i] = G_new[i] - G_old[i];
    }
    *count = keep + 1;
}

/* Returns the number of LS columns kept (0 means C_next = G^t, a plain Lloyd iterate). */
static int aa_mix(const double* dF, const double* dG, int count, int64_t n, int m_t, const double* Gt,
                  const double* Ft, double rank_tol, double* C_next, double* theta_out)
{
    double theta[64];
    if (m_t > count) m_t = count;
    memcpy(C_next, Gt, sizeof(double) * (size_t)n);
    if (m_t <= 0) return 0;
    int rank = orc_ls_qr(dF, n, m_t, Ft, rank_tol, theta);
    for (int j = 0; j < rank; ++j)
        for (int64_t i = 0; i < n; ++i) C_next[i] -= theta[j] * dG[(int64_t)j * n + i];
    if (theta_out)
        for (int j = 0; j < m_t; ++j) theta_out[j] = theta[j];
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
    double* dF = (double*)calloc((size_t)(m > 0 ? m : 1) * n, sizeof(double));
    double* dG = (double*)calloc((size_t)(m > 0 ? m : 1) * n, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * n);
    double* f = (double*)malloc(sizeof(double) * n);
    double* g_old = (double*)malloc(sizeof(double) * n);
    double* f_old = (double*)malloc(sizeof(double) * n);
    int count = 0;
    if (traj) memcpy(traj, x, sizeof(double) * n);
    for (int t = 0; t < iters; ++t) {
        for (int r = 0; r < n; ++r) {
            double s = b[r];
            for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
            g[r] = s;
        }
        for (int r = 0; r < n; ++r) f[r] = g[r] - x[r];
        if (t > 0) hist_push(dF, dG, &count, m, n, g, g_old, f, f_old);
        memcpy(g_old, g, sizeof(double) * n);
        memcpy(f_old, f, sizeof(double) * n);
        int m_t = m < t ? m : t;
        aa_mix(dF, dG, count, n, m_t, g, f, rank_tol, x, NULL);
        if (traj) memcpy(traj + (int64_t)(t + 1) * n, x, sizeof(double) * n);
    }
    free(dF);
    free(dG);
    free(g);
    free(f);
    free(g_old);
    free(f_old);
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

/* The state of Algorithm 1 between two loop passes: everything a pass reads, and what it leaves
 * for the next one.  On entry to pass t: C = C^t (the iterate to assign), CAU = C_AU = G^{t-1},
 * F = F^{t-1}, dF / dG the differences (newest first, `count` of them), Pprev = P^{t-1},
 * E_prev = E^{t-1} and E_prev2 = E^{t-2} (stored energies), m, from_lloyd = whether C^t is a
 * plain Lloyd iterate.  After the pass (unless it terminated): C = C^{t+1}, CAU = G^t, F = F^t,
 * Pprev = P^t, t incremented.  If it terminated, done = 1, C and Pprev hold the result and E
 * its energy. */
typedef struct {
    double* C;
    double* CAU;
    double* F;
    double* dF;           /* m_max x K*d */
    double* dG;
    int32_t* Pprev;       /* N */
    int count;
    int t, m, from_lloyd;
    double E_prev, E_prev2;
    int done;
    double E;             /* energy of the terminal pair */
    int accepted, rejected, assign_passes;
    double theta[64];     /* theta of the last least-squares solve (0 past its rank) */
} orc_state;

static int64_t count_changed(const int32_t* a, const int32_t* b, int64_t N)
{
    int64_t c = 0;
    for (int64_t i = 0; i < N; ++i) c += (a[i] != b[i]);
    return c;
}

/*
 * One loop pass t of Algorithm 1, with the readings:
 *   R3  the revert target C_AU is G^{t-1}, the Lloyd image of the previous stored iterate;
 *   R4, R5  m rule as in orc_m_rule;
 *   R6  the safeguard reverts on E^t >= E^{t-1} (as written);
 *   R7  after a revert the convergence test is applied again;
 *   R8  convergence is only accepted at a Lloyd iterate: if C^t was an accelerated point and
 *       its assignment equals P^{t-1}, the solver reverts to C_AU (= means of P^{t-1}) and
 *       tests again, so the returned C is always the mean of its clusters;
 *   R14 tol > 0 stops when n_changed <= floor(tol * N); tol = 0 is exact equality;
 *   R18 the safeguard is skipped when C^t is itself a Lloyd iterate (reverting would
 *       re-assign the same point; Lloyd's step never increases E).
 * P, G, Fn and Cnext are scratch buffers (N, K*d, K*d, K*d).  rec (optional) gets the pass's
 * trace record.
 */
int orc_step(const double* X, int64_t N, int d, int K, const orc_params* p, orc_state* s, orc_trace* rec_out,
             int32_t* P, double* G, double* Fn, double* Cnext)
{
    const int64_t n = (int64_t)K * d;
    const int64_t thr = p->tol > 0 ? (int64_t)floor(p->tol * (double)N) : 0;
    const int m_max = p->lloyd_only ? 0 : p->m_max;
    const int t = s->t;
    orc_trace rec;
    memset(&rec, 0, sizeof(rec));
    rec.t = t;
    rec.accelerated = !s->from_lloyd;
    rec.margin_lo = rec.margin_hi = NAN;
    /* Check for convergence */
    orc_assign(X, N, d, s->C, K, P, NULL, NULL);
    s->assign_passes++;
    int64_t nch = count_changed(P, s->Pprev, N);
    rec.n_changed = (int)nch;
    int conv = nch <= thr;
    if (conv && s->from_lloyd) {
        double E = orc_energy(X, N, d, s->C, P);
        rec.E_trial = rec.E = E;
        rec.margin_safe = NAN;
        rec.m = s->m;
        if (rec_out) *rec_out = rec;
        s->E = E;
        s->done = 1;
        memcpy(s->Pprev, P, sizeof(int32_t) * (size_t)N);
        return 1;
    }
    /* Adjust the value of m */
    double Et = orc_energy(X, N, d, s->C, P);
    rec.E_trial = Et;
    if (!p->lloyd_only && !p->fixed_m && t >= 3) {
        double num = s->E_prev - Et, den = s->E_prev2 - s->E_prev;
        rec.margin_lo = num - p->eps1 * den;
        rec.margin_hi = num - p->eps2 * den;
    }
    if (!p->lloyd_only && !p->fixed_m)
        s->m = orc_m_rule(s->m, m_max, t, Et, s->E_prev, s->E_prev2, p->eps1, p->eps2);
    rec.m = s->m;
    rec.margin_safe = Et - s->E_prev;
    /* Make sure C^t decreases the energy */
    int reject = !s->from_lloyd && (conv || Et >= s->E_prev);
    if (reject) {
        memcpy(s->C, s->CAU, sizeof(double) * (size_t)n);
        orc_assign(X, N, d, s->C, K, P, NULL, NULL);
        s->assign_passes++;
        s->rejected++;
        rec.rejected = 1;
        Et = orc_energy(X, N, d, s->C, P);
        nch = count_changed(P, s->Pprev, N);
        if (nch <= thr) {
            rec.E = Et;
            if (rec_out) *rec_out = rec;
            s->E = Et;
            s->done = 1;
            memcpy(s->Pprev, P, sizeof(int32_t) * (size_t)N);
            return 1;
        }
    } else if (!s->from_lloyd) {
        s->accepted++;
    }
    rec.E = Et;
    /* Anderson acceleration */
    orc_update(X, N, d, P, K, s->C, G, NULL);
    for (int64_t i = 0; i < n; ++i) Fn[i] = G[i] - s->C[i];
    hist_push(s->dF, s->dG, &s->count, m_max, n, G, s->CAU, Fn, s->F);
    memcpy(s->CAU, G, sizeof(double) * (size_t)n);
    memcpy(s->F, Fn, sizeof(double) * (size_t)n);
    int m_t = s->m < t ? s->m : t;
    rec.m_t = m_t;
    for (int j = 0; j < 64; ++j) s->theta[j] = 0.0;
    int rank = 0;
    if (m_t > 0) {
        rank = aa_mix(s->dF, s->dG, s->count, n, m_t, G, Fn, p->rank_tol, Cnext, s->theta);
    } else {
        memcpy(Cnext, G, sizeof(double) * (size_t)n);
    }
    rec.rank = rank;
    s->from_lloyd = rank == 0;
    s->E_prev2 = s->E_prev;
    s->E_prev = Et;
    memcpy(s->Pprev, P, sizeof(int32_t) * (size_t)N);
    memcpy(s->C, Cnext, sizeof(double) * (size_t)n);
    s->t = t + 1;
    if (rec_out) *rec_out = rec;
    return 0;
}

/*
 * Algorithm 1 (R13: iters = t at termination; Lloyd runs the same loop, so m_max = 0
 * reproduces Lloyd): C^1 = C_AU^1 = G(C^0); F^0 = C^1 - C^0; E^0 = +inf; P^0 = Assign(C^0);
 * then orc_step for t = 1, 2, ... until it terminates or t = max_iter.
 * At max_iter without convergence the returned pair is (P^t, G^t) of the last pass.
 * rho_out (N) and C_out (K*d) are written; trace (optional) gets one record per pass.
 */
int orc_solve(const double* X, int64_t N, int d, int K, const double* C0, const orc_params* p,
              double* C_out, int32_t* rho_out, orc_info* info, orc_trace* trace)
{
    const int64_t n = (int64_t)K * d;
    const int m_max = p->lloyd_only ? 0 : p->m_max;
    const int mm = m_max > 0 ? m_max : 1;
    orc_state s;
    memset(&s, 0, sizeof(s));
    s.C = (double*)malloc(sizeof(double) * (size_t)n);
    s.CAU = (double*)malloc(sizeof(double) * (size_t)n);
    s.F = (double*)malloc(sizeof(double) * (size_t)n);
    s.dF = (double*)calloc((size_t)mm * n, sizeof(double));
    s.dG = (double*)calloc((size_t)mm * n, sizeof(double));
    s.Pprev = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    double* G = (double*)malloc(sizeof(double) * (size_t)n);
    double* Fn = (double*)malloc(sizeof(double) * (size_t)n);
    double* Cnext = (double*)malloc(sizeof(double) * (size_t)n);

    /* C^1 = C_AU^1 = G(C^0); F^0 = C^1 - C^0; E^0 = +inf.  P^0 = Assign(C^0). */
    orc_assign(X, N, d, C0, K, s.Pprev, NULL, NULL);
    s.assign_passes = 1;
    orc_update(X, N, d, s.Pprev, K, C0, G, NULL);
    for (int64_t i = 0; i < n; ++i) s.F[i] = G[i] - C0[i];
    memcpy(s.C, G, sizeof(double) * (size_t)n);
    memcpy(s.CAU, G, sizeof(double) * (size_t)n);
    s.from_lloyd = 1;
    s.E_prev = s.E_prev2 = INFINITY;
    s.m = p->m_init < m_max ? p->m_init : m_max;
    if (s.m < 0) s.m = 0;
    s.t = 1;
    while (s.t <= p->max_iter) {
        const int t = s.t;
        if (orc_step(X, N, d, K, p, &s, trace ? &trace[t - 1] : NULL, P, G, Fn, Cnext)) break;
    }
    orc_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.accepted = s.accepted;
    inf.rejected = s.rejected;
    inf.assign_passes = s.assign_passes;
    if (s.done) {
        inf.iters = s.t;
        inf.converged = 1;
        inf.E = s.E;
        memcpy(C_out, s.C, sizeof(double) * (size_t)n);
        memcpy(rho_out, s.Pprev, sizeof(int32_t) * (size_t)N);
    } else {
        inf.iters = p->max_iter;
        inf.converged = 0;
        memcpy(C_out, s.CAU, sizeof(double) * (size_t)n);
        memcpy(rho_out, s.Pprev, sizeof(int32_t) * (size_t)N);
        inf.E = orc_energy(X, N, d, s.CAU, s.Pprev);
    }
    inf.m_final = s.m;
    if (info) *info = inf;
    free(s.C);
    free(s.CAU);
    free(s.F);
    free(s.dF);
    free(s.dG);
    free(s.Pprev);
    free(P);
    free(G);
    free(Fn);
    free(Cnext);
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
