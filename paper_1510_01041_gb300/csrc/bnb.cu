// bnb.cu -- exact branch-and-bound over slope intervals (sm_103a).
//
// The LMS value is min over slopes s of w(s), the narrowest vertical window
// holding h of the projections z_k(s) = y_k - s x_k (Sec. 3.1).  Any real
// slope s gives an upper bound w(s) >= LMS.  For a slope interval [a, b],
// every z_k(s) lies between lo_k = min(z_k(a), z_k(b)) and hi_k = max(...)
// because z_k is linear in s; order statistics are monotone in each
// argument, so z_(m)(s) >= lo_(m) and z_(m)(s) <= hi_(m) and
//     w(s) >= min over windows a' of lo_(a'+h-1) - hi_(a')
// for every s in [a, b] (a lower bound).  An interval whose lower bound
// exceeds the upper bound strictly cannot contain any slope with w <= the
// upper bound, in particular no optimal slope, and is dropped; ties survive,
// so the lexicographic tie-break over the surviving intervals is unchanged.
// Surviving leaf intervals (single slope buckets of the sweep pipeline) are
// swept exactly, so the answer equals the plain sweep's bit for bit.
//
// Arithmetic: slopes are dyadic, s = K / 2^32 with K a slope key; projections
// are kept as Z_k = z_k * 2^32 = y_k 2^32 - (x_k - xc) K in int64 (guarded to
// |K| < 2^46), xc the midrange of x (a common shift of all projections at a
// fixed slope changes no window width).  Bounds compare in the same units.
//
// The upper bound comes from a few dyadic slopes: the sampled slopes nearest
// a seed slope (a learned prediction) or, without a seed, evenly spaced
// quantiles of the sample, then zoom passes around the best.  Steep and
// unbounded intervals get the bound |s| dh - yr (any h points span at least
// dh in x and at most yr in y); kept buckets holding many events are cut
// into sub-intervals and bounded once more (refinement).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr long long I64_MAX = 0x7fffffffffffffffLL;
constexpr long long K_GUARD = 1LL << 46;

// Set constants of the bounds, into xs[0 .. 2]: the midrange of x (the
// common shift of the projections), dh, a lower bound of the x-span of any
// h points (h points take at least ceil(h / m) distinct integer x, m the
// largest number of points sharing one x, so they span at least that less
// one), and the y range.  The x histogram is kept in shared memory, one half
// of the int16 range at a time.
__global__ void __launch_bounds__(1024) k_x_center(const int *__restrict__ xy, int n, int h, int *__restrict__ xs)
{
    extern __shared__ unsigned s_h[];   // 32768 counters
    __shared__ int s_lo, s_hi, s_ylo, s_yhi;
    __shared__ unsigned s_m;
    if (threadIdx.x == 0) { s_lo = s_ylo = 0x7fffffff; s_hi = s_yhi = -0x7fffffff; s_m = 0u; }
    __syncthreads();
    int lo = 0x7fffffff, hi = -0x7fffffff, ylo = 0x7fffffff, yhi = -0x7fffffff;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        lo = min(lo, px(xy[k]));
        hi = max(hi, px(xy[k]));
        ylo = min(ylo, py(xy[k]));
        yhi = max(yhi, py(xy[k]));
    }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
    atomicMin(&s_ylo, ylo);
    atomicMax(&s_yhi, yhi);
    unsigned m = 0;
    for (int half = 0; half < 2; ++half) {
        for (int k = threadIdx.x; k < 32768; k += blockDim.x) s_h[k] = 0u;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int x = px(xy[k]) + 32768;
            if ((x >> 15) == half) atomicAdd(&s_h[x & 32767], 1u);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 32768; k += blockDim.x) m = max(m, s_h[k]);
        __syncthreads();
    }
    atomicMax(&s_m, m);
    __syncthreads();
    if (threadIdx.x == 0) {
        xs[0] = (int)(((long long)s_lo + s_hi) / 2);
        const unsigned mm = s_m ? s_m : 1u;
        xs[1] = (int)(((unsigned)h + mm - 1u) / mm) - 1;
        xs[2] = s_yhi - s_ylo;
    }
}

// Lower bound of w over slope keys [Klo, Khi] lying wholly on one side of 0
// (steep or unbounded intervals, where the projections at the ends are not
// available): any h points span at least dh in x and at most yr in y, so
// their window at slope s is at least |s| dh - yr; in units of 2^-32,
// |K| dh - yr 2^32 with K the end nearer 0.  0 when the interval contains 0.
__device__ __forceinline__ long long steep_lb(long long Klo, long long Khi, int dh, int yr)
{
    long long K;
    if (Khi <= 0 && Khi > -I64_MAX) K = -Khi;
    else if (Klo >= 0 && Klo < I64_MAX) K = Klo;
    else return 0;
    const __int128 v = (__int128)K * dh - ((__int128)yr << 32);
    if (v <= 0) return 0;
    return v > (__int128)I64_MAX ? I64_MAX : (long long)v;
}

__device__ __forceinline__ long long zscaled(int p, int xc, long long K)
{
    return ((long long)py(p) << 32) - (long long)(px(p) - xc) * K;
}

// CTA-wide minimum and maximum (every thread returns both).
__device__ __forceinline__ void cta_min_max(long long &mn, long long &mx)
{
    __shared__ long long s_mn[32], s_mx[32];
    for (int s = 16; s >= 1; s >>= 1) {
        mn = min(mn, __shfl_xor_sync(FULL, mn, s));
        mx = max(mx, __shfl_xor_sync(FULL, mx, s));
    }
    if ((threadIdx.x & 31) == 0) { s_mn[threadIdx.x >> 5] = mn; s_mx[threadIdx.x >> 5] = mx; }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    mn = s_mn[0];
    mx = s_mx[0];
    for (int w = 1; w < nw; ++w) { mn = min(mn, s_mn[w]); mx = max(mx, s_mx[w]); }
    __syncthreads();
}

// Right shift that brings a span of values below 2^31: 32-bit sort keys
// (v - lo) >> sh leave room for one unit of rounding up.
__device__ __forceinline__ int key_shift(unsigned long long span)
{
    const int bits = span ? 64 - __clzll((long long)span) : 0;
    return bits > 31 ? bits - 31 : 0;
}

// min over windows a of (top[a + h - 1] - bot[a]) for 32-bit keys, reduced over the CTA.
__device__ long long cta_min_window32(const unsigned *top, const unsigned *bot, int n, int h)
{
    __shared__ long long s_red[32];
    long long m = I64_MAX;
    for (int a = threadIdx.x; a + h - 1 < n; a += blockDim.x)
        m = min(m, (long long)top[a + h - 1] - (long long)bot[a]);
    for (int s = 16; s >= 1; s >>= 1) m = min(m, __shfl_xor_sync(FULL, m, s));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? s_red[threadIdx.x] : I64_MAX;
        for (int s = 16; s >= 1; s >>= 1) m = min(m, __shfl_xor_sync(FULL, m, s));
        if (threadIdx.x == 0) s_red[0] = m;
    }
    __syncthreads();
    const long long r = s_red[0];
    __syncthreads();
    return r;
}

// Point sets up to BNB_SMEM_N are sorted whole in shared memory (32-bit
// keys: the words plus merge scratch, 128 KB, or two arrays plus scratch,
// 192 KB, at the limit).  Larger sets are sorted in chunks of BNB_SMEM_N
// keys in shared memory, merged in global scratch.
constexpr int BNB_SMEM_N = 16384;

// Upper bounds: the window width w at dyadic slopes keys[q] (one CTA per
// slope).  In shared memory the projections are sorted as 32-bit keys
// k = (Z - Zmin) >> sh, sh the smallest shift that brings their span below
// 2^31; floor is monotone, so the sorted keys are the shifted order
// statistics, and Z_(a+h-1) - Z_(a) < (k_(a+h-1) - k_(a) + 1) 2^sh.  The
// result is w exactly when sh = 0 and otherwise an upper bound of w larger
// by less than 2^sh units of 2^-32 (a few 10^-5 for slopes of order one),
// which is all an upper bound needs.
__global__ void __launch_bounds__(1024) k_score_dyadic(const int *__restrict__ xy, int n, int h,
                                                       const int *__restrict__ xcp,
                                                       const long long *__restrict__ keys, int nk,
                                                       long long *__restrict__ out,
                                                       long long *__restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int P = 1;
    while (P < n) P <<= 1;
    const bool in_smem = n <= BNB_SMEM_N;
    for (int q = blockIdx.x; q < nk; q += gridDim.x) {
        const long long K = keys[q];
        if (K >= K_GUARD || K <= -K_GUARD) {
            if (threadIdx.x == 0) out[q] = I64_MAX;
            continue;
        }
        const int xc = *xcp;
        long long mn = I64_MAX, mx = -I64_MAX;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const long long z = zscaled(xy[k], xc, K);
            mn = min(mn, z);
            mx = max(mx, z);
        }
        cta_min_max(mn, mx);
        const int sh = key_shift((unsigned long long)(mx - mn));
        unsigned *a = reinterpret_cast<unsigned *>(smem);
        auto key = [&](int k) {
            return k < n ? (unsigned)((unsigned long long)(zscaled(xy[k], xc, K) - mn) >> sh) : 0xffffffffu;
        };
        if (in_smem) {
            const int Ps = P < (int)blockDim.x ? (int)blockDim.x : P;
            cta_fill_merge_sort_any(a, a + Ps, Ps, key);
        } else {
            unsigned *g = reinterpret_cast<unsigned *>(gscratch + (size_t)blockIdx.x * 2 * P);
            a = cta_sort_chunked<BNB_SMEM_N>(a, g, g + P, P, key);
        }
        const long long wk = cta_min_window32(a, a, n, h);
        if (threadIdx.x == 0) out[q] = sh ? (wk + 1) << sh : wk;
        __syncthreads();
    }
}

// Lower bounds of slope intervals [K_lo, K_hi] (keys) and the prune flags.
// In shared memory the hull ends are sorted as 32-bit keys with the shift
// of k_score_dyadic, rounded outward: lo down (floor), hi up (ceil), so
// lo_(a+h-1) - hi_(a) >= (L_(a+h-1) - H_(a)) 2^sh and the bound stays a
// lower bound (exact when sh = 0).
__global__ void __launch_bounds__(1024) k_node_lb(const int *__restrict__ xy, int n, int h,
                                                  const int *__restrict__ xcp,
                                                  const long long *__restrict__ node_keys,
                                                  const int *__restrict__ nnodes_dev,
                                                  const long long *__restrict__ ub,
                                                  unsigned char *__restrict__ prune,
                                                  long long *__restrict__ lb_out,
                                                  long long *__restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int P = 1;
    while (P < n) P <<= 1;
    const bool in_smem = n <= BNB_SMEM_N;
    const int nnodes = *nnodes_dev;
    for (int q = blockIdx.x; q < nnodes; q += gridDim.x) {
        const long long Klo = node_keys[2 * q], Khi = node_keys[2 * q + 1];
        if (Klo <= -K_GUARD || Khi >= K_GUARD || Klo >= K_GUARD || Khi <= -K_GUARD) {
            if (threadIdx.x == 0) {
                const long long lb = steep_lb(Klo, Khi, xcp[1], xcp[2]);
                lb_out[q] = lb;
                prune[q] = lb > *ub ? 1 : 0;
            }
            continue;
        }
        const int xc = *xcp;
        long long mn = I64_MAX, mx = -I64_MAX;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const long long za = zscaled(xy[k], xc, Klo), zb = zscaled(xy[k], xc, Khi);
            mn = min(mn, min(za, zb));
            mx = max(mx, max(za, zb));
        }
        cta_min_max(mn, mx);
        const int sh = key_shift((unsigned long long)(mx - mn));
        const unsigned long long up = (1ull << sh) - 1ull;
        auto klo = [&](int k) {
            if (k >= n) return 0xffffffffu;
            const long long za = zscaled(xy[k], xc, Klo), zb = zscaled(xy[k], xc, Khi);
            return (unsigned)((unsigned long long)(min(za, zb) - mn) >> sh);
        };
        auto khi = [&](int k) {
            if (k >= n) return 0xffffffffu;
            const long long za = zscaled(xy[k], xc, Klo), zb = zscaled(xy[k], xc, Khi);
            return (unsigned)(((unsigned long long)(max(za, zb) - mn) + up) >> sh);
        };
        unsigned *lo = reinterpret_cast<unsigned *>(smem), *hi;
        if (in_smem) {
            const int Ps = P < (int)blockDim.x ? (int)blockDim.x : P;
            hi = lo + Ps;
            cta_fill_merge_sort_any(lo, hi + Ps, Ps, klo);
            cta_fill_merge_sort_any(hi, hi + Ps, Ps, khi);
        } else {
            unsigned *g = reinterpret_cast<unsigned *>(gscratch + (size_t)blockIdx.x * 2 * P);
            unsigned *s = lo;
            lo = cta_sort_chunked<BNB_SMEM_N>(s, g, g + P, P, klo);
            hi = cta_sort_chunked<BNB_SMEM_N>(s, g + 2 * P, g + 3 * P, P, khi);
        }
        long long lb = cta_min_window32(lo, hi, n, h);
        lb = lb < 0 ? 0 : lb << sh;
        if (threadIdx.x == 0) {
            lb_out[q] = lb;
            prune[q] = lb > *ub ? 1 : 0;
        }
        __syncthreads();
    }
}

constexpr unsigned long long BNB_MIN_RANGE = 64;   // events per swept range, at least
#ifndef LMS_PRED_WINDOW
#define LMS_PRED_WINDOW 0.35
#endif
#ifndef LMS_LEARNED_ROUNDS
#define LMS_LEARNED_ROUNDS 2
#endif
constexpr double PRED_WINDOW = LMS_PRED_WINDOW;   // radians around a predicted slope angle

// First index in [0, n) of the sorted array a with a[index] >= key (le =
// false) or a[index] > key (le = true), by a 32-way search: each round every
// lane tests one of 32 evenly spaced splits, so n = 65536 takes four rounds of
// one load per lane instead of sixteen dependent loads.  All lanes of the
// warp call it and get the result.
__device__ __forceinline__ int warp_search(const long long *__restrict__ a, int n, long long key, bool le)
{
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n;   // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) / 32;
        const int at = lo + (lane + 1) * step - 1;
        const bool below = at < hi && (le ? a[at] <= key : a[at] < key);
        const int c = __popc(__ballot_sync(FULL, below));
        lo += c * step;
        hi = min(hi, lo + step);
    }
    const bool below = lo + lane < hi && (le ? a[lo + lane] <= key : a[lo + lane] < key);
    return lo + __popc(__ballot_sync(FULL, below));
}

// Seed slopes.  With a predicted slope: half of them evenly spaced quantiles
// of the sampled slopes whose angle lies within PRED_WINDOW of the
// prediction (the prediction picks the region, the sample finds where pairs
// concentrate in it), half quantiles of all samples.  Without: evenly spaced
// quantiles of all valid samples (mode 0) or the keys of evenly spaced
// angles in (-pi/2, pi/2) (mode 1).  meta[10]: the valid samples.
__global__ void k_pick_seeds(const long long *__restrict__ sorted, const int *__restrict__ meta,
                             const float *__restrict__ pred, int mode, int KS, long long *__restrict__ out)
{
    if (!pred && mode == 1) {
        for (int q = threadIdx.x; q < KS; q += blockDim.x) {
            const double ang = -1.5707963267948966 + 3.141592653589793 * (q + 0.5) / KS;
            const double sp = tan(ang);
            long long k;
            if (sp > 16000.0) k = K_GUARD - 1;
            else if (sp < -16000.0) k = -(K_GUARD - 1);
            else k = (long long)(sp * 4294967296.0);
            out[q] = k;
        }
        return;
    }
    __shared__ int s_lo, s_hi;
    const int m = meta[10];
    if (threadIdx.x < 32) {
        int a = 0, b = m;
        if (pred && m > 0) {
            // the window of slope angles within PRED_WINDOW radians of the prediction
            const double sp = (double)*pred;
            const double ang = (sp == sp) ? atan(sp) : 0.0;
            auto key_of = [](double t) -> long long {
                const double v = tan(t);
                if (v > 16000.0) return K_GUARD - 1;
                if (v < -16000.0) return -(K_GUARD - 1);
                return (long long)(v * 4294967296.0);
            };
            const double half_pi = 1.5707963267948966;
            a = warp_search(sorted, m, key_of(fmax(ang - PRED_WINDOW, -half_pi + 1e-6)), false);
            b = warp_search(sorted, m, key_of(fmin(ang + PRED_WINDOW, half_pi - 1e-6)), true);
            if (b <= a) {                      // no sample in the window: the nearest ones
                a = max(0, min(a, m - 1));
                b = a + 1;
            }
        }
        if (threadIdx.x == 0) { s_lo = a; s_hi = b; }
    }
    __syncthreads();
    const int a = s_lo, b = s_hi;
    // with a prediction the first half of the seeds samples the window and
    // the second half all samples, so a wrong prediction costs nothing
    const int KW = pred ? KS / 2 : KS;
    for (int q = threadIdx.x; q < KS; q += blockDim.x) {
        long long k = I64_MAX;
        if (m > 0) {
            int r;
            if (q < KW) r = a + (int)(((long long)(2 * q + 1) * (b - a)) / (2 * KW));
            else r = (int)(((long long)(2 * (q - KW) + 1) * m) / (2 * (KS - KW)));
            k = sorted[min(r, m - 1)];
        }
        out[q] = k;
    }
}

// Zoom round of the upper bound: KS sample ranks evenly spaced over
// [r* - span, r* + span] around the best seed of the previous round
// (smallest width, ties to the smaller index), r* the rank of its key in the
// sorted sample and span the previous round's spacing of sample ranks
// (round 2: m / KS, m the valid samples; a round 3, when configured:
// 2 span_2 / KS).  The upper
// bound only needs some real slope with a narrow window; narrowing the
// search where the previous round found the narrowest windows brings it
// close to the optimum, and the tighter the bound the fewer slope intervals
// survive.  A round whose previous round found nothing repeats its keys.
__global__ void __launch_bounds__(256) k_zoom_seeds(const long long *__restrict__ sorted,
                                                    const int *__restrict__ meta,
                                                    const long long *__restrict__ prev_keys,
                                                    const long long *__restrict__ prev_w, int KS, int round,
                                                    long long *__restrict__ out)
{
    __shared__ long long s_w[8];
    __shared__ int s_q[8], s_q1, s_r1;
    const int m = meta[10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = threadIdx.x;
    // the best seed: (width, index) minimum over the block
    long long v = q < KS ? prev_w[q] : I64_MAX;
    int idx = v < I64_MAX ? q : -1;
    for (int d = 16; d >= 1; d >>= 1) {
        const long long ov = __shfl_xor_sync(FULL, v, d);
        const int oi = __shfl_xor_sync(FULL, idx, d);
        if (oi >= 0 && (idx < 0 || ov < v || (ov == v && oi < idx))) { v = ov; idx = oi; }
    }
    if (lane == 0) { s_w[warp] = v; s_q[warp] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long bv = I64_MAX;
        int bi = -1;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            if (s_q[k] >= 0 && (bi < 0 || s_w[k] < bv || (s_w[k] == bv && s_q[k] < bi))) { bv = s_w[k]; bi = s_q[k]; }
        s_q1 = bi;
    }
    __syncthreads();
    const int q1 = s_q1;
    if (q1 < 0 || m == 0) {
        if (q < KS) out[q] = prev_keys[q];
        return;
    }
    // its rank in the sample
    if (warp == 0) {
        const int r = warp_search(sorted, m, prev_keys[q1], false);
        if (lane == 0) s_r1 = min(r, m - 1);
    }
    __syncthreads();
    int span = max(1, m / KS);
    for (int k = 2; k < round; ++k) span = max(1, (2 * span + 1) / KS);
    const int r1 = s_r1;
    if (q < KS) {
        const int lo = max(0, r1 - span), hi = min(m, r1 + span + 1);
        const long long len = hi - lo;
        out[q] = sorted[lo + (int)(((2LL * q + 1) * len) / (2LL * KS))];
    }
}

constexpr size_t a256_const(size_t v) { return (v + 255) & ~(size_t)255; }
size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Upper-bound slopes per round (one CTA each, one wave) and rounds: a first
// round of seeds, then a zoom round around the best slope found (a third
// round tightens the bound but costs more than the events it saves).
constexpr int BNB_SEEDS_MAX = 256;
constexpr int BNB_ROUNDS = 2;
constexpr int ROUNDS_MAX = BNB_ROUNDS > LMS_LEARNED_ROUNDS ? BNB_ROUNDS : LMS_LEARNED_ROUNDS;
int bnb_seeds(int sms) { return std::max(64, std::min(BNB_SEEDS_MAX, sms)); }
constexpr int BNB_FIRST_NODES = 128;
// Levels of the interval tree.  The split after the second-to-last level
// makes every child a single bucket, so the last level leaves no node open.
constexpr int BNB_LEVELS = 3;
constexpr int TREE_THREADS = 1024;

// Device-side state of one branch-and-bound fit (read back only for the
// statistics).
struct TreeState {
    int count[2];            // nodes of the current / next level (ping-pong by level parity)
    int evaluated, pruned;   // nodes bounded, nodes dropped
    int levels;              // levels that held nodes
    int kept;                // buckets kept for the exact sweep
    unsigned swept;          // events in the kept buckets
    int covers;              // slope covers handed to the restricted pair pass
    int nruns;               // runs of consecutive kept buckets
    int refine;              // sub-intervals of the refinement level
};

// Page-locked host buffer for the statistics of a fit, one per host thread
// (allocated on first use, kept until the process exits).
unsigned char *host_stage()
{
    thread_local unsigned char *buf = nullptr;
    if (!buf) {
        void *q = nullptr;
        if (cudaHostAlloc(&q, 256, cudaHostAllocPortable) != cudaSuccess) return nullptr;
        buf = static_cast<unsigned char *>(q);
    }
    return buf;
}

// ------------------------------------------------------------ block scans
// Inclusive scan of one value per thread over the CTA (sum or max).
template <bool MAX>
__device__ __forceinline__ long long block_scan(long long v, long long *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long o = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v = MAX ? max(v, o) : v + o;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < nw ? s_warp[lane] : (MAX ? LLONG_MIN : 0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long o = __shfl_up_sync(FULL, t, d);
            if (lane >= d) t = MAX ? max(t, o) : t + o;
        }
        s_warp[lane] = t;
    }
    __syncthreads();
    if (warp > 0) {
        const long long o = s_warp[warp - 1];
        v = MAX ? max(v, o) : v + o;
    }
    __syncthreads();
    return v;
}

// First index in [lo, hi) with a[index] >= t (hi if none).
__device__ __forceinline__ int lower_bound_u(const unsigned *a, int lo, int hi, unsigned long long t)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if ((unsigned long long)a[m] < t) lo = m + 1; else hi = m;
    }
    return lo;
}
// First index in [lo, hi) with a[index] > t (hi if none).
__device__ __forceinline__ int upper_bound_u(const unsigned *a, int lo, int hi, unsigned long long t)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if ((unsigned long long)a[m] <= t) lo = m + 1; else hi = m;
    }
    return lo;
}

__device__ __forceinline__ void node_keys_of(const long long *bnd, int NB, int b0, int b1, long long *keys)
{
    keys[0] = b0 == 0 ? -I64_MAX : bnd[b0 - 1];
    keys[1] = b1 >= NB ? I64_MAX : bnd[b1 - 1];
}

// Exclusive prefix of the sampled pairs per bucket (sbase[NB] = all of them),
// then the first level of the tree: m0 intervals of about equal sampled
// pairs, each at least one bucket.  Interval k ends at f_k =
// min(NB, max(b_k, f_{k-1} + 1)), b_k the first bucket boundary reaching
// k/m0 of the sampled pairs (b_m0 = NB), f_0 = 0; written as a prefix
// maximum, f_k = min(NB, k + max_{j<=k} (b_j - j)).
// It also writes the upper bound: the smallest of the nw seed widths w.
__global__ void __launch_bounds__(TREE_THREADS) k_tree_first(const unsigned *__restrict__ counts,
                                                             const int *__restrict__ meta,
                                                             const long long *__restrict__ bnd, int sms,
                                                             unsigned *__restrict__ sbase, int2 *__restrict__ nodes,
                                                             long long *__restrict__ keys,
                                                             unsigned char *__restrict__ keep,
                                                             TreeState *__restrict__ ts,
                                                             const long long *__restrict__ w, int nw,
                                                             long long *__restrict__ ub)
{
    extern __shared__ unsigned s_base[];   // NB + 1 prefix values, for the searches
    __shared__ long long s_warp[32];
    __shared__ unsigned s_tot;
    {
        long long m = I64_MAX;
        for (int k = threadIdx.x; k < nw; k += blockDim.x) m = min(m, w[k]);
        for (int s = 16; s >= 1; s >>= 1) m = min(m, __shfl_xor_sync(FULL, m, s));
        if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = min(m, s_warp[k]);
            *ub = m;
        }
        __syncthreads();
    }
    const int NB = meta[0] + 1;
    constexpr int PER = BND_MAX / TREE_THREADS;
    // exclusive scan of the counts, PER consecutive buckets per thread
    const int b_beg = threadIdx.x * PER;
    unsigned loc[PER];
    unsigned long long sum = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        loc[r] = b < NB ? counts[b] : 0u;
        sum += loc[r];
    }
    const long long incl = block_scan<false>((long long)sum, s_warp);
    unsigned run = (unsigned)(incl - (long long)sum);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        if (b < NB) sbase[b] = s_base[b] = run;
        run += loc[r];
    }
    if (threadIdx.x == blockDim.x - 1) {
        sbase[NB] = s_base[NB] = (unsigned)incl;
        s_tot = (unsigned)incl;
    }
    for (int b = threadIdx.x; b < NB; b += blockDim.x) keep[b] = 0;
    __syncthreads();
    const unsigned long long E = s_tot;
    const int m0 = min(NB, max(BNB_FIRST_NODES, sms));
    // thread k - 1 computes b_k (k = 1 .. m0; m0 is at most the SM count or 128, below blockDim)
    const int k = threadIdx.x + 1;
    long long v = LLONG_MIN;
    if (k <= m0) {
        int b = lower_bound_u(s_base, 0, NB + 1, E * (unsigned long long)k / (unsigned long long)m0);
        if (k == m0) b = NB;
        v = (long long)b - k;
    }
    // f_k with f_0 = 0 included in the maximum (the j = 0 term is 0)
    long long mx = block_scan<true>(v, s_warp);
    mx = max(mx, 0LL);
    const int f_k = (int)min((long long)NB, mx + k);
    const int f_km1 = __shfl_up_sync(FULL, f_k, 1);
    __shared__ int s_last[32];
    if ((threadIdx.x & 31) == 31) s_last[threadIdx.x >> 5] = f_k;
    __syncthreads();
    const int prev = k == 1 ? 0 : ((threadIdx.x & 31) == 0 ? s_last[(threadIdx.x >> 5) - 1] : f_km1);
    if (k <= m0 && prev < NB) {
        nodes[k - 1] = make_int2(prev, f_k);
        node_keys_of(bnd, NB, prev, f_k, keys + 2 * (k - 1));
    }
    // nodes: every k with f_{k-1} < NB (f is increasing and f_m0 = NB)
    const int is_node = (k <= m0 && prev < NB) ? 1 : 0;
    const long long cnt = block_scan<false>(is_node, s_warp);
    if (threadIdx.x == blockDim.x - 1) {
        ts->count[0] = (int)cnt;
        ts->count[1] = 0;
        ts->evaluated = ts->pruned = ts->levels = ts->kept = 0;
        ts->swept = 0;
        ts->covers = ts->nruns = 0;
    }
}

// One tree step after the bounds of level L: surviving single buckets are
// kept; every other survivor splits into F children of about equal sampled
// pairs (F about fills the SMs at the next level; at the second-to-last
// level every child is a single bucket).  Child boundaries follow
// m'_q = min(max(m_q, m'_{q-1} + 1), b1 - parts + q), m_q the first bucket
// boundary above q/parts of the node's sampled pairs; with u_q = m'_q - q this
// is u_q = max(b0, max_{j<=q} min(m_j - j, b1 - parts)), one warp per node.
__device__ void tree_step_body(int level, int sms, const int *__restrict__ meta,
                                                            const long long *__restrict__ bnd,
                                                            const unsigned *__restrict__ sbase,
                                                            const int2 *__restrict__ cur,
                                                            const unsigned char *__restrict__ prune,
                                                            int2 *__restrict__ nxt, long long *__restrict__ nkeys,
                                                            int *__restrict__ offs,
                                                            unsigned char *__restrict__ keep,
                                                            TreeState *__restrict__ ts)
{
    extern __shared__ unsigned s_base[];   // NB + 1 prefix values, for the searches
    __shared__ long long s_warp[32];
    __shared__ int s_F, s_total;
    const int NB = meta[0] + 1;
    const int nn = ts->count[level & 1];
    if (nn == 0) {
        if (threadIdx.x == 0) ts->count[(level + 1) & 1] = 0;
        return;
    }
    for (int b = threadIdx.x; b <= NB; b += blockDim.x) s_base[b] = sbase[b];
    const bool last_split = level >= BNB_LEVELS - 2;
    // survivors that split, dropped nodes, kept single buckets
    int split = 0, dropped = 0;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const int2 nd = cur[k];
        if (prune[k]) ++dropped;
        else if (nd.y - nd.x == 1) keep[nd.x] = 1;
        else ++split;
    }
    const long long tsplit = block_scan<false>(split, s_warp);
    const long long tdrop = block_scan<false>(dropped, s_warp);
    if (threadIdx.x == blockDim.x - 1) {
        const int S = (int)tsplit;
        s_F = last_split ? 0x7fffffff : (S ? max(2, min(64, sms / S)) : 2);
        ts->evaluated += nn;
        ts->pruned += (int)tdrop;
        ts->levels += nn > 0;
    }
    __syncthreads();
    const int F = s_F;
    // children per node, exclusive offsets (contiguous node chunks per thread)
    const int per = (nn + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per, k1 = min(nn, k0 + per);
    long long csum = 0;
    for (int k = k0; k < k1; ++k) {
        const int2 nd = cur[k];
        csum += (!prune[k] && nd.y - nd.x > 1) ? min(F, nd.y - nd.x) : 0;
    }
    const long long cinc = block_scan<false>(csum, s_warp);
    int o = (int)(cinc - csum);
    for (int k = k0; k < k1; ++k) {
        const int2 nd = cur[k];
        offs[k] = o;
        o += (!prune[k] && nd.y - nd.x > 1) ? min(F, nd.y - nd.x) : 0;
    }
    if (threadIdx.x == blockDim.x - 1) s_total = (int)cinc;
    __syncthreads();
    // children, one warp per splitting node
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nn; k += nw) {
        const int2 nd = cur[k];
        const int len = nd.y - nd.x;
        if (prune[k] || len <= 1) continue;
        const int parts = min(F, len);
        const int C = nd.y - parts;
        const unsigned long long s0 = s_base[nd.x], s1 = s_base[nd.y];
        int carry = nd.x;   // u_{q-1} before the chunk (u_0 = b0)
        int mprev = nd.x;   // m'_{q-1}
        for (int q0 = 1; q0 <= parts; q0 += 32) {
            const int q = q0 + lane;
            int v = INT_MIN;
            if (q <= parts) {
                int m = nd.y;
                if (q < parts) m = upper_bound_u(s_base, nd.x + 1, nd.y, s0 + (s1 - s0) * (unsigned long long)q / parts);
                v = min(m - q, C);
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int ov = __shfl_up_sync(FULL, v, d);
                if (lane >= d) v = max(v, ov);
            }
            const int u = max(carry, v);
            const int mq = u + q;
            int mp = __shfl_up_sync(FULL, mq, 1);
            if (lane == 0) mp = mprev;
            if (q <= parts) {
                const int at = offs[k] + q - 1;
                nxt[at] = make_int2(mp, mq);
                node_keys_of(bnd, NB, mp, mq, nkeys + 2 * at);
            }
            carry = __shfl_sync(FULL, u, 31);
            mprev = __shfl_sync(FULL, mq, 31);
        }
    }
    if (threadIdx.x == 0) ts->count[(level + 1) & 1] = s_total;
}

// ------------------------------------------------------------ sub-bucket refinement
// The last tree level ends at single buckets, and a bucket's lower bound is
// weaker than the bound of a narrower interval by about the spread of the
// projections over the bucket's slope range, which near the optimum (where
// pair slopes crowd) is what keeps most surviving buckets.  So every kept
// interior bucket is cut into F_b sub-intervals of equal key width, each
// bounded once more; the buckets are then replaced by their sub-intervals
// (new boundaries, a keep flag per sub-interval) for the restricted pass
// and the sweep.  F = max(2, SMs / kept) (one wave of bounds), at most
// REFINE_MAX and within the room left under BND_MAX boundaries, and no
// refinement when more than twice the SM count of buckets survive; F_b =
// min(F, the bucket's key width).  Both kernels below derive the same
// F_b and sub-node offsets from the same inputs.
constexpr int REFINE_MAX = 64;
// No refinement when the kept buckets hold fewer events than this (by the
// sampled pairs): a level of bounds costs about as much as sweeping them.
constexpr long long REFINE_MIN_EVENTS = 1 << 16;

struct RefinePlan {
    int F;      // sub-intervals per kept bucket (0: no refinement)
    int total;  // sub-nodes
};

// Per thread: PER consecutive buckets; fb[r] = F_b (0 when the bucket is not cut).
// scount: sampled pairs per bucket (S sampled of emax pairs).
template <int PER>
__device__ RefinePlan refine_plan(const int *__restrict__ meta, const long long *__restrict__ bnd,
                                  const unsigned char *__restrict__ keep, const unsigned *__restrict__ scount,
                                  int S, long long emax, int sms, int (&fb)[PER], int &off, long long *s_warp)
{
    __shared__ int s_F;
    __shared__ long long s_tot;
    const int NB = meta[0] + 1, nbnd = meta[0];
    const int b_beg = threadIdx.x * PER;
    int cut = 0;
    long long smp = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        const bool ok = b > 0 && b < NB - 1 && keep[b] && bnd[b] - bnd[b - 1] >= 2;
        fb[r] = ok ? 1 : 0;
        cut += ok;
        smp += ok ? scount[b] : 0;
    }
    const long long nk = block_scan<false>(cut, s_warp);
    const long long nsmp = block_scan<false>(smp, s_warp);
    if (threadIdx.x == blockDim.x - 1) {
        int F = 0;
        const double est = (double)nsmp * (double)emax / (double)S;   // events in the buckets to cut
        if (nk > 0 && nk <= 2LL * sms && est >= (double)REFINE_MIN_EVENTS) {
            const long long room = (long long)(BND_MAX - 1 - nbnd);
            long long f = max(2LL, (long long)sms / nk);
            f = min(f, 1 + room / nk);
            f = min(f, (long long)REFINE_MAX);
            F = f >= 2 ? (int)f : 0;
        }
        s_F = F;
    }
    __syncthreads();
    const int F = s_F;
    long long sum = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        if (fb[r] && F) fb[r] = (int)min((long long)F, bnd[b] - bnd[b - 1]);
        else fb[r] = 0;
        sum += fb[r];
    }
    const long long inc = block_scan<false>(sum, s_warp);
    off = (int)(inc - sum);
    if (threadIdx.x == blockDim.x - 1) s_tot = inc;
    __syncthreads();
    RefinePlan rp;
    rp.F = F;
    rp.total = (int)s_tot;
    __syncthreads();
    return rp;
}

// Key interval of sub-interval i of the F_b cuts of [lo, hi).
__device__ __forceinline__ long long sub_key(long long lo, long long hi, int i, int Fb)
{
    return lo + (hi - lo) * i / Fb;
}

__device__ void refine_nodes_body(const int *__restrict__ meta,
                                                               const long long *__restrict__ bnd,
                                                               const unsigned char *__restrict__ keep,
                                                               const unsigned *__restrict__ scount, int S,
                                                               long long emax, int sms,
                                                               long long *__restrict__ nkeys,
                                                               TreeState *__restrict__ ts)
{
    __shared__ long long s_warp[32];
    constexpr int PER = BND_MAX / TREE_THREADS;
    int fb[PER], off;
    const RefinePlan rp = refine_plan<PER>(meta, bnd, keep, scount, S, emax, sms, fb, off, s_warp);
    const int b_beg = threadIdx.x * PER;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        if (!fb[r]) continue;
        const int b = b_beg + r;
        const long long lo = bnd[b - 1], hi = bnd[b];
        for (int i = 0; i < fb[r]; ++i) {
            nkeys[2 * (off + i)] = sub_key(lo, hi, i, fb[r]);
            nkeys[2 * (off + i) + 1] = sub_key(lo, hi, i + 1, fb[r]);
        }
        off += fb[r];
    }
    if (threadIdx.x == 0) ts->refine = rp.total;
}

// Replace the buckets by their sub-intervals: boundaries and keep flags into
// the scratch arrays, then copied over bnd (padded with I64_MAX to the new
// power of two) and keep, and the new counts into meta.
__device__ void refine_apply_body(int *__restrict__ meta, long long *__restrict__ bnd,
                                                               unsigned char *__restrict__ keep,
                                                               const unsigned char *__restrict__ prune,
                                                               const unsigned *__restrict__ scount, int S,
                                                               long long emax, int sms,
                                                               long long *__restrict__ bnd_tmp,
                                                               unsigned char *__restrict__ keep_tmp,
                                                               TreeState *__restrict__ ts)
{
    __shared__ long long s_warp[32];
    __shared__ int s_nb;
    constexpr int PER = BND_MAX / TREE_THREADS;
    int fb[PER], off;
    const RefinePlan rp = refine_plan<PER>(meta, bnd, keep, scount, S, emax, sms, fb, off, s_warp);
    if (rp.total == 0) return;
    const int NB = meta[0] + 1;
    const int b_beg = threadIdx.x * PER;
    // new buckets per old bucket: F_b when cut, else 1
    long long cnt = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) cnt += (b_beg + r < NB) ? (fb[r] ? fb[r] : 1) : 0;
    const long long inc = block_scan<false>(cnt, s_warp);
    if (threadIdx.x == blockDim.x - 1) s_nb = (int)inc;
    int o = (int)(inc - cnt);
    int pr = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        if (b >= NB) break;
        if (fb[r]) {
            const long long lo = bnd[b - 1], hi = bnd[b];
            for (int i = 0; i < fb[r]; ++i) {
                const bool drop = prune[off + i] != 0;
                pr += drop;
                keep_tmp[o + i] = drop ? 0 : 1;
                bnd_tmp[o + i] = i + 1 < fb[r] ? sub_key(lo, hi, i + 1, fb[r]) : hi;
            }
            off += fb[r];
            o += fb[r];
        } else {
            keep_tmp[o] = keep[b];
            if (b < NB - 1) bnd_tmp[o] = bnd[b];
            ++o;
        }
    }
    const long long pruned = block_scan<false>(pr, s_warp);
    const int NB2 = s_nb, nbnd2 = NB2 - 1;
    int P2 = 1;
    while (P2 <= nbnd2) P2 <<= 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) bnd[k] = k < nbnd2 ? bnd_tmp[k] : I64_MAX;
    for (int k = threadIdx.x; k < NB2; k += blockDim.x) keep[k] = keep_tmp[k];
    if (threadIdx.x == blockDim.x - 1) {
        ts->evaluated += rp.total;
        ts->pruned += (int)pruned;
        ts->levels += 1;
        meta[0] = nbnd2;
        meta[1] = P2;
    }
}

// Covers of the runs of kept buckets for the restricted pair pass: bucket
// b holds keys [bnd[b - 1], bnd[b]), a key being floor(slope 2^32).  At most
// PRE_MAX covers: the runs are grouped at the PRE_MAX - 1 widest gaps
// between neighbouring runs (the same grouping as merging the closest
// neighbours one at a time; gaps measured in slope); each cover is the key
// range from its first run's start to its last run's end.  Unused entries
// are empty ranges.
__device__ void tree_covers_body(const int *__restrict__ meta,
                                                              const long long *__restrict__ bnd,
                                                              const unsigned char *__restrict__ keep,
                                                              int *__restrict__ runs, long long *__restrict__ cov,
                                                              TreeState *__restrict__ ts)
{
    __shared__ long long s_warp[32];
    __shared__ int s_R, s_sep[PRE_MAX];
    __shared__ double s_gv[32];
    __shared__ int s_gi[32];
    const int NB = meta[0] + 1;
    constexpr int PER = BND_MAX / TREE_THREADS;
    const int b_beg = threadIdx.x * PER;
    int starts = 0, kept = 0;
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        if (b < NB && keep[b]) {
            ++kept;
            starts += (b == 0 || !keep[b - 1]);
        }
    }
    const long long kinc = block_scan<false>(kept, s_warp);
    const long long sinc = block_scan<false>(starts, s_warp);
    int at = (int)(sinc - starts);
    for (int r = 0; r < PER; ++r) {
        const int b = b_beg + r;
        if (b < NB && keep[b] && (b == 0 || !keep[b - 1])) {
            int e = b + 1;
            while (e < NB && keep[e]) ++e;
            runs[2 * at] = b;
            runs[2 * at + 1] = e;
            ++at;
        }
    }
    if (threadIdx.x == blockDim.x - 1) {
        s_R = (int)sinc;
        ts->kept = (int)kinc;
        ts->nruns = (int)sinc;
    }
    __syncthreads();
    const int R = s_R;
    auto lo_of = [&](int r) -> double {
        const int b = runs[2 * r];
        if (b == 0) return -INFINITY;
        const double v = (double)bnd[b - 1] * 0x1p-32;
        return v - (fabs(v) * 0x1p-18 + 0x1p-30);
    };
    auto hi_of = [&](int r) -> double {
        const int e = runs[2 * r + 1];
        if (e >= NB) return (double)INFINITY;
        const double v = (double)bnd[e - 1] * 0x1p-32;
        return v + (fabs(v) * 0x1p-18 + 0x1p-30);
    };
    // separators: the PRE_MAX - 1 widest gaps (gap r lies between runs r - 1 and r)
    const int nsep = min(R - 1, PRE_MAX - 1);
    // with at most PRE_MAX runs every run is a cover of its own
    if (R <= PRE_MAX)
        for (int t = threadIdx.x; t < nsep; t += blockDim.x) s_sep[t] = t + 1;
    for (int t = 0; t < (R <= PRE_MAX ? 0 : nsep); ++t) {
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int r = 1 + threadIdx.x; r < R; r += blockDim.x) {
            bool taken = false;
            for (int u = 0; u < t; ++u) taken |= s_sep[u] == r;
            if (taken) continue;
            const double g = lo_of(r) - hi_of(r - 1);
            if (g > bv || (g == bv && r < bi)) { bv = g; bi = r; }
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            const double ov = __shfl_xor_sync(FULL, bv, d);
            const int oi = __shfl_xor_sync(FULL, bi, d);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { s_gv[threadIdx.x >> 5] = bv; s_gi[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = -1.0;
            int vi = 0x7fffffff;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (s_gv[w] > v || (s_gv[w] == v && s_gi[w] < vi)) { v = s_gv[w]; vi = s_gi[w]; }
            s_sep[t] = vi;
        }
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // separators in increasing order
        int sep[PRE_MAX];
        for (int t = 0; t < nsep; ++t) sep[t] = s_sep[t];
        for (int a = 1; a < nsep; ++a)
            for (int b = a; b > 0 && sep[b - 1] > sep[b]; --b) { const int tt = sep[b]; sep[b] = sep[b - 1]; sep[b - 1] = tt; }
        // cover: the key range from the first bucket of its first run to the
        // end of its last run (-inf / +inf at the outer buckets)
        int nc = 0;
        if (R == 0) {
            cov[0] = -I64_MAX;   // nothing kept: every pair
            cov[1] = I64_MAX;
            nc = 1;
        } else {
            int first = 0;
            for (int t = 0; t <= nsep; ++t) {
                const int last = t < nsep ? sep[t] - 1 : R - 1;
                const int b0 = runs[2 * first], e1 = runs[2 * last + 1];
                cov[2 * nc] = b0 == 0 ? -I64_MAX : bnd[b0 - 1];
                cov[2 * nc + 1] = e1 >= NB ? I64_MAX : bnd[e1 - 1];
                ++nc;
                first = last + 1;
            }
        }
        for (int c = nc; c < PRE_MAX; ++c) cov[2 * c] = cov[2 * c + 1] = I64_MAX;   // empty
        ts->covers = nc;
    }
}

// The tree kernels.  The last tree step also plans the refinement (its
// sub-intervals' keys into rkeys, their number into ts->refine); the covers
// kernel first applies it (the bounds of the sub-intervals are computed
// between the two), so the refinement costs no launches of its own.
__global__ void __launch_bounds__(TREE_THREADS) k_tree_step(int level, int sms, const int *__restrict__ meta,
                                                            const long long *__restrict__ bnd,
                                                            const unsigned *__restrict__ sbase,
                                                            const int2 *__restrict__ cur,
                                                            const unsigned char *__restrict__ prune,
                                                            int2 *__restrict__ nxt, long long *__restrict__ nkeys,
                                                            int *__restrict__ offs,
                                                            unsigned char *__restrict__ keep,
                                                            TreeState *__restrict__ ts,
                                                            const unsigned *__restrict__ scount, int S,
                                                            long long emax, long long *__restrict__ rkeys)
{
    tree_step_body(level, sms, meta, bnd, sbase, cur, prune, nxt, nkeys, offs, keep, ts);
    if (level == BNB_LEVELS - 1) {
        __syncthreads();
        refine_nodes_body(meta, bnd, keep, scount, S, emax, sms, rkeys, ts);
    }
}

__global__ void __launch_bounds__(TREE_THREADS) k_tree_covers(int *__restrict__ meta, long long *__restrict__ bnd,
                                                              unsigned char *__restrict__ keep,
                                                              const unsigned char *__restrict__ prune,
                                                              const unsigned *__restrict__ scount, int S,
                                                              long long emax, int sms,
                                                              long long *__restrict__ bnd_tmp,
                                                              unsigned char *__restrict__ keep_tmp,
                                                              int *__restrict__ runs, long long *__restrict__ cov,
                                                              TreeState *__restrict__ ts)
{
    refine_apply_body(meta, bnd, keep, prune, scount, S, emax, sms, bnd_tmp, keep_tmp, ts);
    __syncthreads();
    tree_covers_body(meta, bnd, keep, runs, cov, ts);
}

// Sweep ranges over the kept events (after the restricted count: base holds
// the kept buckets' event starts): the kept events of each maximal run of
// kept buckets are cut into pieces of about `target` events (a range never
// spans a dropped bucket: the kinetic order must see every event between its
// first and last slope); k_snap_ranges then moves every bound to the next
// start of a group of equal slopes.  A range costs one start sort of all n
// points (about a wave of start sorts per SM count of ranges) plus its events
// one after another, so R ranges of K kept events take about
// (R / SMs) T_sort + (K / R) T_event; with T_sort / T_event about 128
// events' worth at 152 SMs that is least near K / R = sqrt(0.8 K) events per
// range.  At least BNB_MIN_RANGE events per range, at least total / G (the
// caller passes the SM count: one wave of start sorts) and at most W ranges.
__global__ void __launch_bounds__(TREE_THREADS) k_tree_ranges(const int *__restrict__ meta,
                                                              const unsigned *__restrict__ base,
                                                              const int *__restrict__ runs, int W, int G,
                                                              unsigned *__restrict__ range,
                                                              TreeState *__restrict__ ts)
{
    __shared__ long long s_warp[32];
    __shared__ long long s_cnt;
    const int NB = meta[0] + 1;
    const unsigned total = base[NB];
    const int nr = ts->nruns;
    // run lengths, RPT per thread (strided), then the smallest target of the
    // form t0 2^k whose pieces number at most W
    constexpr int RPT = (BND_MAX + 1) / TREE_THREADS + 1;
    unsigned len[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int r = threadIdx.x + i * TREE_THREADS;
        len[i] = r < nr ? base[runs[2 * r + 1]] - base[runs[2 * r]] : 0u;
    }
    unsigned long long t = max((unsigned long long)BNB_MIN_RANGE, (unsigned long long)sqrt(0.8 * (double)total));
    t = max(t, ((unsigned long long)total + G - 1) / G);
    for (;;) {
        long long c = 0;
#pragma unroll
        for (int i = 0; i < RPT; ++i) c += (long long)((len[i] + t - 1) / t);
        c = block_scan<false>(c, s_warp);
        if (threadIdx.x == blockDim.x - 1) s_cnt = c;
        __syncthreads();
        const long long cnt = s_cnt;
        __syncthreads();
        if (cnt <= (long long)W) break;
        t *= 2;
    }
    if (threadIdx.x == 0) ts->swept = total;
    // pieces per run, exclusive offsets (runs in chunks per thread)
    const int per = (nr + blockDim.x - 1) / blockDim.x;
    const int r0 = threadIdx.x * per, r1 = min(nr, r0 + per);
    long long psum = 0;
    for (int r = r0; r < r1; ++r) {
        const unsigned len = base[runs[2 * r + 1]] - base[runs[2 * r]];
        psum += (long long)((len + t - 1) / t);
    }
    const long long pinc = block_scan<false>(psum, s_warp);
    __shared__ long long s_pieces;
    if (threadIdx.x == blockDim.x - 1) s_pieces = pinc;
    long long o = pinc - psum;
    for (int r = r0; r < r1; ++r) {
        const unsigned a = base[runs[2 * r]], len = base[runs[2 * r + 1]] - a;
        const unsigned long long pieces = (len + t - 1) / t;
        for (unsigned long long q = 0; q < pieces; ++q) {
            range[2 * o] = a + (unsigned)(len * q / pieces);
            range[2 * o + 1] = a + (unsigned)(len * (q + 1) / pieces);
            ++o;
        }
    }
    __syncthreads();
    // the ranges past the last piece are empty
    for (long long w = s_pieces + threadIdx.x; w < W; w += blockDim.x) {
        range[2 * w] = total;
        range[2 * w + 1] = total;
    }
}

size_t bnb_extra_bytes(int n, int sms)
{
    int P = 1;
    while (P < n) P <<= 1;
    const int grid = 2 * sms;
    size_t b = 0;
    b += a256(64);                                   // xc, ub
    b += a256((size_t)BNB_SEEDS_MAX * ROUNDS_MAX * 8 * 2);   // seed keys, seed widths of every round
    b += a256(sizeof(TreeState));                    // tree state
    b += 2 * a256((size_t)BND_MAX * sizeof(int2));   // nodes, two levels
    b += 2 * a256((size_t)BND_MAX * 2 * 8);          // node keys, two levels
    b += a256((size_t)BND_MAX);                      // prune flags
    b += a256((size_t)BND_MAX * 8);                  // node lower bounds
    b += a256((size_t)BND_MAX * 4);                  // child offsets
    b += a256((size_t)BND_MAX);                      // keep mask
    b += a256((size_t)BND_MAX * 4);                  // sampled pairs per bucket
    b += a256((size_t)(BND_MAX + 1) * 4);            // their prefix
    b += a256((size_t)(BND_MAX + 1) * 2 * 4);        // runs of kept buckets
    b += a256((size_t)PRE_MAX * 2 * 8);              // key ranges of the kept covers
    b += band_scratch_bytes(n);                      // restricted count: sorted words per cover
    b += (n > BNB_SMEM_N) ? a256((size_t)grid * 2 * P * 8) : 0;   // chunked sorts: four key arrays per CTA
    return b;
}

// The whole branch-and-bound is queued on the stream without a host round
// trip: seeds and upper bound, BNB_LEVELS levels of interval bounds with
// their splits, the slope covers of the kept buckets, the restricted pair
// pass, the sweep ranges, the exact sweep of the kept events and the argmin.
// Levels left without nodes cost two empty launches.  With stats the call
// waits for the fit to read them back; without, it returns at once.
int run_bnb(const SweepPlan &p, const short *x, const short *y, const float *pred_dev, int seed_mode, lms_result *out,
            lms_bnb_stats *stats, void *extra, int sms, cudaStream_t st, cudaEvent_t pred_ready)
{
    const int n = p.n, h = p.h;
    unsigned char *cur = static_cast<unsigned char *>(extra);
    auto take = [&](size_t bytes) { void *r = cur; cur += a256(bytes); return r; };
    int *xc = (int *)take(64);
    long long *ub = (long long *)(xc + 4);
    const int KS = bnb_seeds(sms);
    long long *seed_keys = (long long *)take((size_t)BNB_SEEDS_MAX * ROUNDS_MAX * 8 * 2);
    long long *seed_w = seed_keys + (size_t)KS * ROUNDS_MAX;
    TreeState *ts = (TreeState *)take(sizeof(TreeState));
    int2 *nodes[2];
    nodes[0] = (int2 *)take((size_t)BND_MAX * sizeof(int2));
    nodes[1] = (int2 *)take((size_t)BND_MAX * sizeof(int2));
    long long *nkeys[2];
    nkeys[0] = (long long *)take((size_t)BND_MAX * 2 * 8);
    nkeys[1] = (long long *)take((size_t)BND_MAX * 2 * 8);
    unsigned char *prune = (unsigned char *)take(BND_MAX);
    long long *lbv = (long long *)take((size_t)BND_MAX * 8);
    int *offs = (int *)take((size_t)BND_MAX * 4);
    unsigned char *keep = (unsigned char *)take(BND_MAX);
    unsigned *scount = (unsigned *)take((size_t)BND_MAX * 4);
    unsigned *sbase = (unsigned *)take((size_t)(BND_MAX + 1) * 4);
    int *runs = (int *)take((size_t)(BND_MAX + 1) * 2 * 4);
    long long *cov = (long long *)take((size_t)PRE_MAX * 2 * 8);
    void *band_scr = take(band_scratch_bytes(n));
    int P = 1;
    while (P < n) P <<= 1;
    long long *gscr = (n > BNB_SMEM_N) ? (long long *)take((size_t)2 * sms * 2 * P * 8) : nullptr;
    const int grid = 2 * sms;

    if (launch_sweep_sample(p, x, y, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (launch_sample_counts(p, scount, st) != cudaSuccess) return LMS_ERR_CUDA;
    {
        StageTimer _t(STAGE_SEEDS, st);
        cudaFuncSetAttribute(k_x_center, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 * 4);
        k_x_center<<<1, 1024, 32768 * 4, st>>>(p.xy, n, h, xc);
    }
    if (pred_ready && cudaStreamWaitEvent(st, pred_ready, 0) != cudaSuccess) return LMS_ERR_CUDA;
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_pick_seeds<<<1, 128, 0, st>>>(sorted_sample(p), p.meta, pred_dev, seed_mode, KS, seed_keys);
    }
    const int Ps = P < 1024 ? 1024 : P;   // the shared-memory sorts fill whole 1024-thread CTAs
    // 32-bit keys: one sorted array plus merge scratch; two sorted arrays plus scratch
    const size_t one_sort = (n <= BNB_SMEM_N) ? (size_t)2 * Ps * 4 : (size_t)2 * BNB_SMEM_N * 4;
    const size_t two_sorts = (n <= BNB_SMEM_N) ? (size_t)3 * Ps * 4 : (size_t)2 * BNB_SMEM_N * 4;
    cudaFuncSetAttribute(k_score_dyadic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_sort);
    cudaFuncSetAttribute(k_node_lb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)two_sorts);
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_score_dyadic<<<std::min(KS, grid), 1024, one_sort, st>>>(p.xy, n, h, xc, seed_keys, KS, seed_w, gscr);
    }
    const int rounds = pred_dev ? LMS_LEARNED_ROUNDS : BNB_ROUNDS;
    for (int r = 2; r <= rounds; ++r) {
        long long *keys_r = seed_keys + (size_t)(r - 1) * KS, *w_r = seed_w + (size_t)(r - 1) * KS;
        {
            StageTimer _t(STAGE_SEEDS, st);
            k_zoom_seeds<<<1, 256, 0, st>>>(sorted_sample(p), p.meta, keys_r - KS, w_r - KS, KS, r, keys_r);
        }
        {
            StageTimer _t(STAGE_SEEDS, st);
            k_score_dyadic<<<std::min(KS, grid), 1024, one_sort, st>>>(p.xy, n, h, xc, keys_r, KS, w_r, gscr);
        }
    }
    // the interval tree, level by level, all on the device
    const size_t tree_smem = (size_t)(BND_MAX + 1) * sizeof(unsigned);
    cudaFuncSetAttribute(k_tree_first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tree_smem);
    cudaFuncSetAttribute(k_tree_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tree_smem);
    {
        StageTimer _t(STAGE_TREE, st);
        k_tree_first<<<1, TREE_THREADS, tree_smem, st>>>(scount, p.meta, p.bnd, sms, sbase, nodes[0], nkeys[0], keep,
                                                          ts, seed_w, KS * rounds, ub);
    }
    // the refinement's sub-interval keys: the last level's input keys, consumed
    // by its bounds before the last tree step writes them
    long long *rkeys = nkeys[(BNB_LEVELS - 1) & 1];
    for (int L = 0; L < BNB_LEVELS; ++L) {
        {
            StageTimer _t(STAGE_NODE_LB, st);
            k_node_lb<<<sms, 1024, two_sorts, st>>>(p.xy, n, h, xc, nkeys[L & 1], &ts->count[L & 1], ub, prune, lbv,
                                                    gscr);
        }
        {
            StageTimer _t(STAGE_TREE, st);
            k_tree_step<<<1, TREE_THREADS, tree_smem, st>>>(L, sms, p.meta, p.bnd, sbase, nodes[L & 1], prune,
                                                            nodes[(L + 1) & 1], nkeys[(L + 1) & 1], offs, keep, ts,
                                                            scount, p.S, p.emax, rkeys);
        }
    }
    {
        // the kept buckets' sub-intervals (planned by the last tree step) bounded
        StageTimer _t(STAGE_NODE_LB, st);
        k_node_lb<<<sms, 1024, two_sorts, st>>>(p.xy, n, h, xc, rkeys, &ts->refine, ub, prune, lbv, gscr);
    }
    {
        // refinement applied (lbv and offs, no longer needed, hold the new
        // boundaries and flags meanwhile), then the covers
        StageTimer _t(STAGE_TREE, st);
        k_tree_covers<<<1, TREE_THREADS, 0, st>>>(p.meta, p.bnd, keep, prune, scount, p.S, p.emax, sms, lbv,
                                                  reinterpret_cast<unsigned char *>(offs), runs, cov, ts);
    }
    // exact events of the kept buckets only: p.base becomes their starts
    if (launch_sweep_count(p, keep, cov, band_scr, stats != nullptr, st) != cudaSuccess) return LMS_ERR_CUDA;
    {
        StageTimer _t(STAGE_PLAN, st);
        // at least kept / SMs events a range: one wave of start sorts
        k_tree_ranges<<<1, TREE_THREADS, 0, st>>>(p.meta, p.base, runs, p.W, std::min(p.G, sms), p.range, ts);
    }
    if (launch_sweep_finish(p, keep, st, false, true) != cudaSuccess) return LMS_ERR_CUDA;
    if (launch_argmin(p.cands, p.W + p.G, out, LMS_ALGO_BNB, p.meta + 3, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return LMS_ERR_CUDA;
    if (stats) {
        unsigned char *hs = host_stage();
        if (!hs) return LMS_ERR_CUDA;
        if (cudaMemcpyAsync(hs, ts, sizeof(TreeState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hs + 64, p.meta, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hs + 128, ub, sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return LMS_ERR_CUDA;
        TreeState t;
        std::memcpy(&t, hs, sizeof(t));
        const int *meta = reinterpret_cast<const int *>(hs + 64);
        long long ubh;
        std::memcpy(&ubh, hs + 128, sizeof(ubh));
        stats->events_total = (unsigned)meta[5];
        stats->events_swept = t.swept;
        stats->buckets_total = meta[0] + 1;
        stats->buckets_swept = t.kept;
        stats->nodes_evaluated = t.evaluated;
        stats->nodes_pruned = t.pruned;
        stats->levels = t.levels;
        stats->seeded = pred_dev ? 1 : 0;
        stats->upper_bound = ubh == I64_MAX ? -1.0 : (double)ubh / 4294967296.0;
    }
    return LMS_OK;
}

}  // namespace lms
