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
// quantiles of the sample.
#include <cuda_runtime.h>

#include <algorithm>
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

__global__ void k_x_center(const int *__restrict__ xy, int n, int *__restrict__ xc)
{
    __shared__ int s_lo, s_hi;
    if (threadIdx.x == 0) { s_lo = 0x7fffffff; s_hi = -0x7fffffff; }
    __syncthreads();
    int lo = 0x7fffffff, hi = -0x7fffffff;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        lo = min(lo, px(xy[k]));
        hi = max(hi, px(xy[k]));
    }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
    __syncthreads();
    if (threadIdx.x == 0) *xc = (int)(((long long)s_lo + s_hi) / 2);
}

__device__ void cta_bitonic_i64(long long *a, int P)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const long long x0 = a[i], x1 = a[l];
                if ((x0 > x1) == up) { a[i] = x1; a[l] = x0; }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ long long zscaled(int p, int xc, long long K)
{
    return ((long long)py(p) << 32) - (long long)(px(p) - xc) * K;
}

// min over windows of (hiarr[a + h - 1] - loarr[a]) with a reduction over the CTA.
__device__ long long cta_min_window(const long long *top, const long long *bot, int n, int h)
{
    __shared__ long long s_red[32];
    long long m = I64_MAX;
    for (int a = threadIdx.x; a + h - 1 < n; a += blockDim.x) m = min(m, top[a + h - 1] - bot[a]);
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

// Upper bounds: exact w at dyadic slopes keys[q] (one CTA per slope).
__global__ void __launch_bounds__(1024) k_score_dyadic(const int *__restrict__ xy, int n, int h,
                                                       const int *__restrict__ xcp,
                                                       const long long *__restrict__ keys, int nk,
                                                       long long *__restrict__ out,
                                                       long long *__restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int P = 1;
    while (P < n) P <<= 1;
    const bool in_smem = n <= SORT_SMEM_N;
    for (int q = blockIdx.x; q < nk; q += gridDim.x) {
        const long long K = keys[q];
        if (K >= K_GUARD || K <= -K_GUARD) {
            if (threadIdx.x == 0) out[q] = I64_MAX;
            continue;
        }
        long long *a = in_smem ? reinterpret_cast<long long *>(smem) : gscratch + (size_t)blockIdx.x * 2 * P;
        const int xc = *xcp;
        auto z = [&](int k) { return k < n ? zscaled(xy[k], xc, K) : I64_MAX; };
        const int Ps = P < (int)blockDim.x ? (int)blockDim.x : P;
        if (!in_smem || !cta_fill_merge_sort_any(a, a + Ps, Ps, z)) {
            for (int k = threadIdx.x; k < P; k += blockDim.x) a[k] = z(k);
            __syncthreads();
            cta_bitonic_i64(a, P);
        }
        const long long w = cta_min_window(a, a, n, h);
        if (threadIdx.x == 0) out[q] = w;
        __syncthreads();
    }
}

// Lower bounds of slope intervals [K_lo, K_hi] (keys) and the prune flags.
__global__ void __launch_bounds__(1024) k_node_lb(const int *__restrict__ xy, int n, int h,
                                                  const int *__restrict__ xcp,
                                                  const long long *__restrict__ node_keys, int nnodes,
                                                  const long long *__restrict__ ub,
                                                  unsigned char *__restrict__ prune,
                                                  long long *__restrict__ lb_out,
                                                  long long *__restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int P = 1;
    while (P < n) P <<= 1;
    const bool in_smem = n <= SORT_SMEM_N;
    for (int q = blockIdx.x; q < nnodes; q += gridDim.x) {
        const long long Klo = node_keys[2 * q], Khi = node_keys[2 * q + 1];
        if (Klo <= -K_GUARD || Khi >= K_GUARD || Klo >= K_GUARD || Khi <= -K_GUARD) {
            if (threadIdx.x == 0) { prune[q] = 0; lb_out[q] = 0; }
            continue;
        }
        const int Ps = (in_smem && P < (int)blockDim.x) ? (int)blockDim.x : P;
        long long *lo = in_smem ? reinterpret_cast<long long *>(smem) : gscratch + (size_t)blockIdx.x * 2 * P;
        long long *hi = lo + Ps;
        const int xc = *xcp;
        auto zlo = [&](int k) {
            return k < n ? min(zscaled(xy[k], xc, Klo), zscaled(xy[k], xc, Khi)) : I64_MAX;
        };
        auto zhi = [&](int k) {
            return k < n ? max(zscaled(xy[k], xc, Klo), zscaled(xy[k], xc, Khi)) : I64_MAX;
        };
        if (!in_smem || !cta_fill_merge_sort_any(lo, hi + Ps, Ps, zlo) ||
            !cta_fill_merge_sort_any(hi, hi + Ps, Ps, zhi)) {
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                lo[k] = zlo(k);
                hi[k] = zhi(k);
            }
            __syncthreads();
            cta_bitonic_i64(lo, P);
            cta_bitonic_i64(hi, P);
        }
        long long lb = cta_min_window(lo, hi, n, h);
        if (lb < 0) lb = 0;
        if (threadIdx.x == 0) {
            lb_out[q] = lb;
            prune[q] = lb > *ub ? 1 : 0;
        }
        __syncthreads();
    }
}

__global__ void k_min_ub(const long long *__restrict__ w, int nk, long long *__restrict__ ub)
{
    long long m = I64_MAX;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) m = min(m, w[k]);
    for (int s = 16; s >= 1; s >>= 1) m = min(m, __shfl_xor_sync(FULL, m, s));
    if (threadIdx.x == 0) *ub = m;
}

#ifndef LMS_BNB_MIN_RANGE
#define LMS_BNB_MIN_RANGE 512
#endif
constexpr unsigned long long BNB_MIN_RANGE = LMS_BNB_MIN_RANGE;   // events per swept range, at least
constexpr double PRED_WINDOW = 0.35;   // radians around a predicted slope angle

// Seed slopes.  With a predicted slope: half of them evenly spaced quantiles
// of the sampled slopes whose angle lies within PRED_WINDOW of the
// prediction (the prediction picks the region, the sample finds where pairs
// concentrate in it), half quantiles of all samples.  Without: evenly spaced
// quantiles of all valid samples (mode 0) or the keys of evenly spaced
// angles in (-pi/2, pi/2) (mode 1).
__global__ void k_pick_seeds(const long long *__restrict__ sorted, int S, const float *__restrict__ pred,
                             int mode, int KS, long long *__restrict__ out)
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
    __shared__ int s_m, s_lo, s_hi;
    if (threadIdx.x == 0) {
        int lo = 0, hi = S;
        while (lo < hi) { int m = (lo + hi) >> 1; if (sorted[m] < I64_MAX) lo = m + 1; else hi = m; }
        s_m = lo;
        int a = 0, b = s_m;
        if (pred && s_m > 0) {
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
            const long long klo = key_of(fmax(ang - PRED_WINDOW, -half_pi + 1e-6));
            const long long khi = key_of(fmin(ang + PRED_WINDOW, half_pi - 1e-6));
            int x0 = 0, x1 = s_m;
            while (x0 < x1) { int m = (x0 + x1) >> 1; if (sorted[m] < klo) x0 = m + 1; else x1 = m; }
            a = x0;
            x1 = s_m;
            while (x0 < x1) { int m = (x0 + x1) >> 1; if (sorted[m] <= khi) x0 = m + 1; else x1 = m; }
            b = x0;
            if (b <= a) {                      // no sample in the window: the nearest ones
                a = max(0, min(a, s_m - 1));
                b = a + 1;
            }
        }
        s_lo = a;
        s_hi = b;
    }
    __syncthreads();
    const int m = s_m, a = s_lo, b = s_hi;
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

constexpr size_t a256_const(size_t v) { return (v + 255) & ~(size_t)255; }
size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Page-locked host staging for the device-to-host reads of a fit, so that
// they are queued asynchronously and waited for once.  One buffer per host
// thread, allocated on first use and kept for the life of the process (a fit
// waits for its reads before it returns, so nothing is in flight between
// fits).  Layout: meta (8 ints), upper bound, bucket counts, boundaries,
// kept-bucket starts, prune flags.
constexpr size_t HS_META = 0, HS_UB = 32, HS_CNT = 64;
constexpr size_t HS_BND = HS_CNT + (size_t)BND_MAX * 4;
constexpr size_t HS_KBASE = HS_BND + (size_t)BND_MAX * 8;
constexpr size_t HS_PRUNE = HS_KBASE + a256_const((size_t)(BND_MAX + 1) * 4);
constexpr size_t HS_BYTES = HS_PRUNE + (size_t)BND_MAX;

unsigned char *host_stage()
{
    thread_local unsigned char *buf = nullptr;
    if (!buf) {
        void *q = nullptr;
        if (cudaHostAlloc(&q, HS_BYTES, cudaHostAllocPortable) != cudaSuccess) return nullptr;
        buf = static_cast<unsigned char *>(q);
    }
    return buf;
}

}  // namespace

constexpr int BNB_SEEDS = 64;
constexpr int BNB_FIRST_NODES = 128;

size_t bnb_extra_bytes(int n, int sms)
{
    int P = 1;
    while (P < n) P <<= 1;
    const int grid = 2 * sms;
    size_t b = 0;
    b += a256(64);                                   // xc, ub
    b += a256((size_t)BNB_SEEDS * 8 * 2);            // seed keys, seed widths
    b += a256((size_t)BND_MAX * 2 * 8);              // node keys
    b += a256((size_t)BND_MAX);                      // prune flags
    b += a256((size_t)BND_MAX * 8);                  // node lower bounds
    b += a256((size_t)BND_MAX);                      // keep mask
    b += a256((size_t)BND_MAX * 4);                  // sampled pairs per bucket
    b += a256((size_t)PRE_MAX * sizeof(float2));     // slope pre-filter of the restricted pair passes
    b += (n > SORT_SMEM_N) ? a256((size_t)grid * 2 * P * 8) : 0;
    return b;
}

// Host-driven B&B: the bucket counts decide the tree, the device evaluates
// bounds level by level.  Synchronises with the stream between levels.
int run_bnb(const SweepPlan &p, const short *x, const short *y, const float *pred_dev, int seed_mode, lms_result *out,
            lms_bnb_stats *stats, void *extra, int sms, cudaStream_t st)
{
    const int n = p.n, h = p.h;
    unsigned char *cur = static_cast<unsigned char *>(extra);
    auto take = [&](size_t bytes) { void *r = cur; cur += a256(bytes); return r; };
    int *xc = (int *)take(64);
    long long *ub = (long long *)(xc + 4);
    long long *seed_keys = (long long *)take((size_t)BNB_SEEDS * 8 * 2);
    long long *seed_w = seed_keys + BNB_SEEDS;
    long long *node_keys = (long long *)take((size_t)BND_MAX * 2 * 8);
    unsigned char *prune = (unsigned char *)take(BND_MAX);
    long long *lbv = (long long *)take((size_t)BND_MAX * 8);
    unsigned char *keep = (unsigned char *)take(BND_MAX);
    unsigned *scount = (unsigned *)take((size_t)BND_MAX * 4);
    float2 *pre = (float2 *)take((size_t)PRE_MAX * sizeof(float2));
    int P = 1;
    while (P < n) P <<= 1;
    long long *gscr = (n > SORT_SMEM_N) ? (long long *)take((size_t)2 * sms * 2 * P * 8) : nullptr;
    const int grid = 2 * sms;

    unsigned char *hs = host_stage();
    if (!hs) return LMS_ERR_CUDA;
    int *h_meta = reinterpret_cast<int *>(hs + HS_META);
    long long *h_ub = reinterpret_cast<long long *>(hs + HS_UB);
    const unsigned *cnt = reinterpret_cast<const unsigned *>(hs + HS_CNT);
    const long long *bnd = reinterpret_cast<const long long *>(hs + HS_BND);
    const unsigned *kbase = reinterpret_cast<const unsigned *>(hs + HS_KBASE);
    unsigned char *h_prune = hs + HS_PRUNE;

    if (launch_sweep_sample(p, x, y, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (launch_sample_counts(p, scount, st) != cudaSuccess) return LMS_ERR_CUDA;
    // bucket structure to the host; the tree weighs buckets by sampled pairs
    // (the buckets are quantile ranges of the sample), so no pass over all
    // pairs is needed before the bounds have pruned.  The reads are waited
    // for after the seed stage is queued, so the host builds the first level
    // while the GPU scores the seeds.
    cudaEvent_t sampled;
    if (cudaEventCreateWithFlags(&sampled, cudaEventDisableTiming) != cudaSuccess) return LMS_ERR_CUDA;
    const bool queued = cudaMemcpyAsync(h_meta, p.meta, sizeof(int) * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                        cudaMemcpyAsync(hs + HS_CNT, scount, sizeof(unsigned) * BND_MAX, cudaMemcpyDeviceToHost,
                                        st) == cudaSuccess &&
                        cudaMemcpyAsync(hs + HS_BND, p.bnd, sizeof(long long) * BND_MAX, cudaMemcpyDeviceToHost,
                                        st) == cudaSuccess &&
                        cudaEventRecord(sampled, st) == cudaSuccess;
    if (!queued) {
        cudaEventDestroy(sampled);
        return LMS_ERR_CUDA;
    }
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_x_center<<<1, 1024, 0, st>>>(p.xy, n, xc);
    }
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_pick_seeds<<<1, 128, 0, st>>>(sorted_sample(p), p.S, pred_dev, seed_mode, BNB_SEEDS, seed_keys);
    }
    const int Ps = P < 1024 ? 1024 : P;   // the shared-memory sorts fill whole 1024-thread CTAs
    // one sorted array plus merge scratch; two sorted arrays plus scratch
    const size_t one_sort = (n <= SORT_SMEM_N) ? (size_t)2 * Ps * 8 : 0;
    const size_t two_sorts = (n <= SORT_SMEM_N) ? (size_t)3 * Ps * 8 : 0;
    cudaFuncSetAttribute(k_score_dyadic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_sort);
    cudaFuncSetAttribute(k_node_lb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)two_sorts);
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_score_dyadic<<<std::min(BNB_SEEDS, grid), 1024, one_sort, st>>>(p.xy, n, h, xc, seed_keys, BNB_SEEDS,
                                                                           seed_w, gscr);
    }
    {
        StageTimer _t(STAGE_SEEDS, st);
        k_min_ub<<<1, 32, 0, st>>>(seed_w, BNB_SEEDS, ub);
    }
    const cudaError_t waited = cudaEventSynchronize(sampled);
    cudaEventDestroy(sampled);
    if (waited != cudaSuccess) return LMS_ERR_CUDA;
    const int NB = h_meta[0] + 1;
    std::vector<unsigned> base(NB + 1);
    base[0] = 0;
    for (int b = 0; b < NB; ++b) base[b + 1] = base[b] + cnt[b];
    const unsigned E = base[NB];
    std::vector<unsigned char> keepv(NB, 0);
    // first level: equal-event ranges of buckets
    struct Node { int b0, b1; };
    std::vector<Node> nodes;
    {
        const int m0 = std::min(NB, std::max(BNB_FIRST_NODES, sms));
        int prev = 0;
        for (int k = 1; k <= m0; ++k) {
            const unsigned long long target = (unsigned long long)E * k / m0;
            int b = (int)(std::lower_bound(base.begin(), base.begin() + NB + 1, (unsigned)target) - base.begin());
            if (k == m0) b = NB;
            b = std::max(b, prev + 1);
            if (b > NB) b = NB;
            if (b > prev) nodes.push_back({prev, b});
            prev = b;
            if (prev >= NB) break;
        }
    }
    long long evaluated = 0, pruned = 0;
    int levels = 0;
    std::vector<long long> hk;
    std::vector<unsigned char> hp;
    while (!nodes.empty()) {
        ++levels;
        const int nn = (int)nodes.size();
        hk.resize(2 * nn);
        for (int k = 0; k < nn; ++k) {
            hk[2 * k] = nodes[k].b0 == 0 ? -I64_MAX : bnd[nodes[k].b0 - 1];
            hk[2 * k + 1] = nodes[k].b1 >= NB ? I64_MAX : bnd[nodes[k].b1 - 1];
        }
        for (int off = 0; off < nn; off += BND_MAX) {
            const int chunk = std::min(BND_MAX, nn - off);
            if (cudaMemcpyAsync(node_keys, hk.data() + 2 * off, sizeof(long long) * 2 * chunk, cudaMemcpyHostToDevice,
                                st) != cudaSuccess)
                return LMS_ERR_CUDA;
            {
                StageTimer _t(STAGE_NODE_LB, st);
                k_node_lb<<<std::min(chunk, grid), 1024, two_sorts, st>>>(p.xy, n, h, xc, node_keys, chunk, ub, prune,
                                                                        lbv, gscr);
            }
            hp.resize(nn);
            if (cudaMemcpyAsync(h_prune, prune, chunk, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                return LMS_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return LMS_ERR_CUDA;
            std::memcpy(hp.data() + off, h_prune, chunk);
        }
        evaluated += nn;
        // survivors split into F children of about equal sampled events, F
        // chosen so that the next level about fills the SMs (fewer levels,
        // each a host round trip)
        int split = 0;
        for (int k = 0; k < nn; ++k)
            if (!hp[k] && nodes[k].b1 - nodes[k].b0 > 1) ++split;
        const int F = split ? std::max(2, std::min(16, sms / split)) : 2;
        std::vector<Node> next;
        for (int k = 0; k < nn; ++k) {
            const Node nd = nodes[k];
            if (hp[k]) { ++pruned; continue; }
            if (nd.b1 - nd.b0 == 1) { keepv[nd.b0] = 1; continue; }
            const int parts = std::min(F, nd.b1 - nd.b0);
            int prev_b = nd.b0;
            for (int q = 1; q <= parts; ++q) {
                int m = nd.b1;
                if (q < parts) {
                    const unsigned long long tgt =
                        base[nd.b0] + (unsigned long long)(base[nd.b1] - base[nd.b0]) * q / parts;
                    m = (int)(std::upper_bound(base.begin() + prev_b + 1, base.begin() + nd.b1, (unsigned)tgt) -
                              base.begin());
                    m = std::min(std::max(m, prev_b + 1), nd.b1 - (parts - q));
                }
                next.push_back({prev_b, m});
                prev_b = m;
            }
        }
        nodes.swap(next);
    }
    // slope covers of the runs of kept buckets for the pair passes: bucket b
    // holds keys [bnd[b - 1], bnd[b]), a key being floor(slope 2^32); each
    // cover is widened by more than the float slope error (2^-21 relative)
    // and rounded outward; at most PRE_MAX covers (closest runs merged)
    std::vector<std::pair<double, double>> cov;
    unsigned kept_buckets = 0;
    for (int b = 0; b < NB;) {
        if (!keepv[b]) { ++b; continue; }
        int e = b + 1;
        while (e < NB && keepv[e]) ++e;
        kept_buckets += (unsigned)(e - b);
        const double lo = b == 0 ? -INFINITY : (double)bnd[b - 1] * 0x1p-32;
        const double hi = e >= NB ? INFINITY : (double)bnd[e - 1] * 0x1p-32;
        cov.push_back({lo - (std::isinf(lo) ? 0.0 : std::fabs(lo) * 0x1p-18 + 0x1p-30),
                       hi + (std::isinf(hi) ? 0.0 : std::fabs(hi) * 0x1p-18 + 0x1p-30)});
        b = e;
    }
    while (cov.size() > (size_t)PRE_MAX) {
        size_t best = 1;
        for (size_t k = 2; k < cov.size(); ++k)
            if (cov[k].first - cov[k - 1].second < cov[best].first - cov[best - 1].second) best = k;
        cov[best - 1].second = cov[best].second;
        cov.erase(cov.begin() + best);
    }
    // rounded outward to floats; covers that now touch or overlap are merged
    // so that they stay sorted and disjoint (the device searches them)
    std::vector<float2> prev;
    for (size_t k = 0; k < cov.size(); ++k) {
        float2 f;
        f.x = std::nextafter((float)cov[k].first, -INFINITY);
        f.y = std::nextafter((float)cov[k].second, INFINITY);
        if (!prev.empty() && f.x <= prev.back().y) prev.back().y = std::max(prev.back().y, f.y);
        else prev.push_back(f);
    }
    const int npre = (int)prev.size();
    if (cudaMemcpyAsync(keep, keepv.data(), NB, cudaMemcpyHostToDevice, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (npre > 0 && cudaMemcpyAsync(pre, prev.data(), sizeof(float2) * npre, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    // exact events of the kept buckets only: p.base becomes their starts
    if (launch_sweep_count(p, keep, npre > 0 ? pre : nullptr, npre, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (cudaMemcpyAsync(hs + HS_KBASE, p.base, sizeof(unsigned) * (NB + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(h_meta, p.meta, sizeof(int) * 6, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_ub, ub, sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LMS_ERR_CUDA;
    const unsigned events_total = (unsigned)h_meta[5];
    const long long ub_host = *h_ub;
    const unsigned run = kbase[NB];
    // ranges: pieces of about `target` events inside each run of consecutive
    // kept buckets (a range never spans a dropped bucket: the kinetic order
    // must see every event between its first and last slope); the device
    // then moves every bound forward to the next start of a group of equal
    // slopes.  About one range per sweeping warp, but at least
    // BNB_MIN_RANGE events each, so that a range's start sort pays off.
    std::vector<unsigned> rng(2 * (size_t)p.W, 0u);
    {
        std::vector<std::pair<unsigned, unsigned>> runs;
        for (int b = 0; b < NB;) {
            if (!keepv[b] || kbase[b + 1] == kbase[b]) { ++b; continue; }
            int e = b + 1;
            while (e < NB && keepv[e]) ++e;
            runs.push_back({kbase[b], kbase[e]});
            b = e;
        }
        unsigned long long target = std::max<unsigned long long>(BNB_MIN_RANGE, ((unsigned long long)run + p.G - 1) / p.G);
        for (;;) {
            unsigned long long count = 0;
            for (const auto &r : runs) count += (r.second - r.first + target - 1) / target;
            if (count <= (unsigned long long)p.W) break;
            target *= 2;
        }
        size_t used = 0;
        for (const auto &r : runs) {
            const unsigned long long len = r.second - r.first;
            const unsigned long long pieces = (len + target - 1) / target;
            for (unsigned long long k = 0; k < pieces; ++k) {
                rng[2 * used] = r.first + (unsigned)(len * k / pieces);
                rng[2 * used + 1] = r.first + (unsigned)(len * (k + 1) / pieces);
                ++used;
            }
        }
        for (size_t w = used; w < (size_t)p.W; ++w) { rng[2 * w] = run; rng[2 * w + 1] = run; }
    }
    if (cudaMemcpyAsync(p.range, rng.data(), sizeof(unsigned) * 2 * p.W, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    if (launch_sweep_finish(p, keep, st, false, npre > 0 ? pre : nullptr, npre) != cudaSuccess) return LMS_ERR_CUDA;
    if (launch_argmin(p.cands, p.W + p.G, out, LMS_ALGO_BNB, p.meta + 3, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LMS_ERR_CUDA;
    if (stats) {
        stats->events_total = events_total;
        stats->events_swept = run;
        stats->buckets_total = NB;
        stats->buckets_swept = kept_buckets;
        stats->nodes_evaluated = evaluated;
        stats->nodes_pruned = pruned;
        stats->levels = levels;
        stats->seeded = pred_dev ? 1 : 0;
        stats->upper_bound = ub_host == I64_MAX ? -1.0 : (double)ub_host / 4294967296.0;
    }
    return LMS_OK;
}

}  // namespace lms
