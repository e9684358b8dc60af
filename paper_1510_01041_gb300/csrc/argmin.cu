// argmin.cu -- deterministic final reduction and translation to the primal
// line (Algorithm 1: the parallel reduction over the bracelets and the map
// back to the primal plane, Sec. 3.4).
//
// Candidates are ordered by the exact lexicographic key (w, theta1, theta2,
// i, j), a total order, so the winner does not depend on the reduction
// order.  The winning slope is reduced by gcd; theta1, theta2 and med_sq are
// each a single correctly rounded double operation on exact integers.
#include "common.cuh"
#include "kernels.cuh"

namespace lms {

namespace {

__device__ __forceinline__ long long gcd_ll(long long a, long long b)
{
    while (b) { long long r = a % b; a = b; b = r; }
    return a;
}

__global__ void __launch_bounds__(1024) k_argmin(const Cand *__restrict__ cands, int count,
                                                 lms_result *__restrict__ out, int algorithm,
                                                 const int *__restrict__ err)
{
    __shared__ Cand s_best[32];
    Cand best = cand_empty();
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        const Cand c = cands[k];
        if (cand_better(c, best)) best = c;
    }
    best = warp_best(best);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (warp != 0) return;
    best = lane < (int)(blockDim.x >> 5) ? s_best[lane] : cand_empty();
    best = warp_best(best);
    if (lane != 0) return;
    lms_result r;
    r.algorithm = algorithm;
    if (best.dx <= 0) {
        r.w_num = r.w_den = r.s_num = r.s_den = r.t_num = r.t_den = 0;
        r.theta1 = r.theta2 = r.med_sq = 0.0;
        r.i = r.j = -1;
        r.status = LMS_ERR_INTERNAL;
        *out = r;
        return;
    }
    const long long dx = best.dx, dy = best.dy;
    long long g = gcd_ll(dy < 0 ? -dy : dy, dx);
    if (g <= 0) g = 1;
    r.s_num = dy / g;
    r.s_den = dx / g;
    r.w_num = best.w / g;
    r.w_den = r.s_den;
    r.t_num = best.t / g;
    r.t_den = 2 * r.s_den;
    r.theta1 = __ddiv_rn((double)r.s_num, (double)r.s_den);
    r.theta2 = __ddiv_rn((double)r.t_num, (double)r.t_den);
    const double half = __ddiv_rn((double)r.w_num, (double)(2 * r.w_den));
    r.med_sq = __dmul_rn(half, half);
    r.i = best.i;
    r.j = best.j;
    r.status = (best.i < 0) ? LMS_ERR_VERTICAL : LMS_OK;
    // err points at the sweep's error word; err[4] / err[5] are the events
    // its ranges covered and the events there were: every event must be
    // swept exactly once
    if (err && (*err || err[4] != err[5])) r.status = LMS_ERR_INTERNAL;
    *out = r;
}

}  // namespace

cudaError_t launch_argmin(const Cand *cands, int count, lms_result *out, int algorithm, const int *err,
                          cudaStream_t st)
{
    StageTimer _t(STAGE_ARGMIN, st);
    k_argmin<<<1, 1024, 0, st>>>(cands, count, out, algorithm, err);
    return cudaGetLastError();
}

}  // namespace lms
