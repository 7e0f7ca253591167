// Head of Algorithm 1 (device side), shared by the low-d pass and the dense assignment chain.
// Runs in one thread after the fixed-order reduction of the pass's energy and change count.
#pragma once

#include "km_internal.cuh"

namespace km {

// After P^t = Assign(C^t): convergence test, dynamic m, energy safeguard.
//   Reading R4: m is only adjusted once E^{t-2} is finite (t >= 3).
//   Reading R5: the ratio test is written without the division.
//   Reading R6: equality reverts.  Reading R8: a converged accelerated point is confirmed by
//   reverting to C_AU.  Also the hard iteration guard and the non-finite input status.
//   fixed_m: the fixed-m strategy of Section 3 (Tab. 2), m never changes.
__device__ __forceinline__ void controller_trial(SolveState* st, double E, long long nch, long long thr,
                                                 int lloyd_only, int fixed_m, double eps1, double eps2,
                                                 int m_max, int max_iter)
{
    st->body_runs += 1;
    if (st->status != KM_OK || st->body_runs > (unsigned)max_iter + 2u) {
        if (st->status == KM_OK) st->status = KM_ETIMEOUT;
        st->done = 1;
        return;
    }
    st->passes += 1;
    st->n_changed = nch;
    st->E_trial = E;
    const bool conv = nch <= thr;
    if (conv && st->from_lloyd) {                  // converged at a Lloyd iterate: return
        st->done = 1;
        st->converged = 1;
        st->E_cur = E;
        st->E_final = E;
        st->final_src = 0;
        return;
    }
    if (!lloyd_only && !fixed_m && st->t >= 3) {
        const double num = st->E_prev - E, den = st->E_prev2 - st->E_prev;
        if (num < eps1 * den)
            st->m = st->m - 1 > 0 ? st->m - 1 : 0;
        else if (num > eps2 * den)
            st->m = st->m + 1 < m_max ? st->m + 1 : m_max;
    }
    const bool reject = !st->from_lloyd && (conv || E >= st->E_prev);
    if (reject) {
        st->revert = 1;
    } else {
        st->revert = 0;
        if (!st->from_lloyd) st->accepted += 1;
        st->E_cur = E;
    }
}

// After the revert pass P^t = Assign(C_AU): bookkeeping and the convergence test again (R7).
__device__ __forceinline__ void controller_revert(SolveState* st, double E, long long nch, long long thr)
{
    st->passes += 1;
    st->rejected += 1;
    st->n_changed = nch;
    st->E_cur = E;
    if (nch <= thr) {
        st->done = 1;
        st->converged = 1;
        st->E_final = E;
        st->final_src = 1;
    }
}

}  // namespace km
