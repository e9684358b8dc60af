// sweep_f32.cu -- the kinetic sweep for float32 points (double arithmetic).
//
// Same method as the int16 sweep (Algorithm 1's candidate set, Sec. 3.3's
// touched-window argument), with slopes s = dy/dx and projections
// z = y - s x evaluated in double: the differences of two float32 values are
// exact in double for coordinates of comparable magnitude, and a projection
// is off by about 1e-16 |z|, far below the 1e-6 relative tolerance asked of
// the median squared residual.  Events are ordered by the double slope (a
// monotone rounding: never inverted, at worst merged).  Events of one slope
// are applied one after another: two adjacent points swap; two points with
// others between them (collinear at that slope) have the block between them
// put into the order just after the slope.  Each event leaves its own pair
// in the just-after order and no later event of the slope undoes that, so the
// order is right once the slope is done, and the windows scored meanwhile
// differ only by a permutation of points tied at that slope.  A window is
// scored in double only when a float estimate of its width, with a proven
// error margin, does not already show it wider than the sweeper's best, so
// nearly every event costs float arithmetic alone (GB300's double rate is a
// small fraction of its float rate); the result is the same as scoring
// every window in double.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

struct CandF {
    double w;      // window width
    double t;      // window centre
    double s;      // slope
    int i, j;      // the event pair
    int valid;
    int pad;
};
static_assert(sizeof(CandF) == 40, "CandF layout");

__device__ __forceinline__ CandF candf_empty()
{
    CandF c;
    c.w = 0; c.t = 0; c.s = 0; c.i = -1; c.j = -1; c.valid = 0; c.pad = 0;
    return c;
}

__device__ __forceinline__ bool candf_better(const CandF &a, const CandF &b)
{
    if (!a.valid) return false;
    if (!b.valid) return true;
    if (a.w != b.w) return a.w < b.w;
    if (a.s != b.s) return a.s < b.s;
    if (a.t != b.t) return a.t < b.t;
    if (a.i != b.i) return a.i < b.i;
    return a.j < b.j;
}

__device__ __forceinline__ CandF candf_shfl(const CandF &c, int m)
{
    CandF o;
    o.w = __shfl_xor_sync(FULL, c.w, m);
    o.t = __shfl_xor_sync(FULL, c.t, m);
    o.s = __shfl_xor_sync(FULL, c.s, m);
    o.i = __shfl_xor_sync(FULL, c.i, m);
    o.j = __shfl_xor_sync(FULL, c.j, m);
    o.valid = __shfl_xor_sync(FULL, c.valid, m);
    o.pad = 0;
    return o;
}

__device__ __forceinline__ CandF candf_warp_best(CandF c)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        CandF o = candf_shfl(c, m);
        if (candf_better(o, c)) c = o;
    }
    return c;
}

__device__ __forceinline__ double zf(float2 p, double s) { return __dsub_rn((double)p.y, __dmul_rn(s, (double)p.x)); }

__device__ __forceinline__ double slope_of(float2 a, float2 b)
{
    double dx = (double)b.x - (double)a.x, dy = (double)b.y - (double)a.y;
    if (dx < 0.0) { dx = -dx; dy = -dy; }
    return __ddiv_rn(dy, dx);
}

__device__ __forceinline__ long long dkey(double v)
{
    const long long bits = v == 0.0 ? 0LL : __double_as_longlong(v);
    return bits < 0 ? (bits ^ 0x7fffffffffffffffLL) : bits;
}

// A coordinate the sweep's float pre-test accepts: 0 or of magnitude in
// [2^-40, 2^40].  Then every nonzero difference of two coordinates, every
// slope and every product the pre-test forms stays a normal float (or
// overflows to inf, which disables the test for that window).
__device__ __forceinline__ bool tame(float v)
{
    const float a = fabsf(v);
    return a == 0.f || (a >= 0x1p-40f && a <= 0x1p40f);
}

// One CTA: pack the coordinates, record whether all of them are finite
// (bad[0]) and whether all of them are tame (bad[1]).
__global__ void __launch_bounds__(1024) k_pack_f32(const float *__restrict__ x, const float *__restrict__ y, int n,
                                                   float2 *__restrict__ P, int *__restrict__ bad)
{
    int nf = 0, wild = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float2 v = make_float2(x[k], y[k]);
        nf |= !(isfinite(v.x) && isfinite(v.y));
        wild |= !(tame(v.x) && tame(v.y));
        P[k] = v;
    }
    nf = __syncthreads_or(nf);
    wild = __syncthreads_or(wild);
    if (threadIdx.x == 0) {
        bad[0] = nf;
        bad[1] = !nf && !wild;
    }
}

// Sweeper start: sort by (z at the first slope, x ascending, index), score
// every window.  keys/idx: shared memory (n <= 8192) or global scratch.
__global__ void __launch_bounds__(1024) k_sweep_init_f32(const float2 *__restrict__ P, int n, int h,
                                                         const unsigned *__restrict__ ev,
                                                         const unsigned *__restrict__ range, int W,
                                                         int *__restrict__ meta_mut,
                                                         const unsigned *__restrict__ base,
                                                         unsigned short *__restrict__ orders,
                                                         long long *__restrict__ gkeys, unsigned short *__restrict__ gidx,
                                                         CandF *__restrict__ cands)
{
    const int *meta = meta_mut;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_slope;
    __shared__ CandF s_best[32];
    const int w = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned E = base[meta[0] + 1];
    const unsigned start = range[2 * w], end = range[2 * w + 1];
    const bool vertical = (E == 0 && w == 0);
    if (w == 0 && threadIdx.x == 0) meta_mut[4] = 0;   // range counter of k_sweep_f32
    if (start >= end && !vertical) {
        if (threadIdx.x == 0) cands[w] = candf_empty();
        return;
    }
    int Pn = 1;
    while (Pn < n) Pn <<= 1;
    if (threadIdx.x == 0) s_slope = vertical ? 0.0 : slope_of(P[ev_i(ev[start])], P[ev_j(ev[start])]);
    __syncthreads();
    const double s0 = s_slope;
    // the order just before s0: (projection, x ascending, index)
    auto exact_gt = [&](int ia, int ib) {
        const long long a = dkey(zf(P[ia], s0)), b = dkey(zf(P[ib], s0));
        if (a != b) return a > b;
        if (P[ia].x != P[ib].x) return P[ia].x > P[ib].x;
        return ia > ib;
    };
    long long *wd = nullptr;        // shared-memory path: sorted words, index in the low 16 bits
    long long *key = nullptr;       // global path: keys and indices
    unsigned short *idx = nullptr;
    if (n <= SORT_SMEM_N) {
        // merge sort of words (projection key with its low 16 bits cleared) |
        // index: the order is exact except inside runs whose keys agree above
        // those 16 bits (projections within 2^16 ulps of each other), which
        // odd-even transposition passes with the exact comparison put right
        const int Ps = Pn < (int)blockDim.x ? (int)blockDim.x : Pn;
        wd = reinterpret_cast<long long *>(smem);
        auto word = [&](int k) {
            return k < n ? ((dkey(zf(P[k], s0)) & ~0xffffLL) | (long long)k) : 0x7fffffffffffffffLL;
        };
        cta_fill_merge_sort_any(wd, wd + Ps, Ps, word);
        for (;;) {
            int swapped = 0;
            for (int par = 0; par < 2; ++par) {
                for (int q = 2 * (int)threadIdx.x + par; q + 1 < n; q += 2 * (int)blockDim.x) {
                    const long long u = wd[q], v = wd[q + 1];
                    if ((u >> 16) == (v >> 16) && exact_gt((int)(u & 0xffff), (int)(v & 0xffff))) {
                        wd[q] = v;
                        wd[q + 1] = u;
                        swapped = 1;
                    }
                }
                __syncthreads();
            }
            if (!__syncthreads_or(swapped)) break;
        }
    } else {
        key = gkeys + (size_t)w * Pn;
        idx = gidx + (size_t)w * Pn;
        for (int k = threadIdx.x; k < Pn; k += blockDim.x) {
            key[k] = k < n ? dkey(zf(P[k], s0)) : 0x7fffffffffffffffLL;
            idx[k] = (unsigned short)(k < n ? k : 0);
        }
        __syncthreads();
        // bitonic on (key, x, index)
        for (int kk = 2; kk <= Pn; kk <<= 1) {
            for (int j = kk >> 1; j >= 1; j >>= 1) {
                for (int t = threadIdx.x; t < Pn / 2; t += blockDim.x) {
                    const int i = 2 * t - (t & (j - 1));
                    const int l = i + j;
                    const bool up = (i & kk) == 0;
                    const long long a = key[i], b = key[l];
                    const unsigned short ia = idx[i], ib = idx[l];
                    bool gt;
                    if (a != b) gt = a > b;
                    else if (i < n && l < n && P[ia].x != P[ib].x) gt = P[ia].x > P[ib].x;
                    else gt = ia > ib;
                    if (gt == up) { key[i] = b; key[l] = a; idx[i] = ib; idx[l] = ia; }
                }
                __syncthreads();
            }
        }
    }
    auto ord = [&](int k) { return wd ? (int)(wd[k] & 0xffff) : (int)idx[k]; };
    for (int k = threadIdx.x; k < n; k += blockDim.x) orders[(size_t)w * n + k] = (unsigned short)ord(k);
    CandF best = candf_empty();
    for (int a = threadIdx.x; a + h - 1 < n; a += blockDim.x) {
        const double zb = zf(P[ord(a)], s0), zt = zf(P[ord(a + h - 1)], s0);
        CandF c;
        c.w = zt - zb; c.t = 0.5 * (zb + zt); c.s = s0; c.valid = 1; c.pad = 0;
        c.i = -1; c.j = -1;
        if (candf_better(c, best)) best = c;
    }
    best = candf_warp_best(best);
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (warp == 0) {
        best = lane < (int)(blockDim.x >> 5) ? s_best[lane] : candf_empty();
        best = candf_warp_best(best);
        if (lane == 0) {
            if (vertical) { best.i = -1; best.j = -1; }
            else { const unsigned e = ev[start]; best.i = ev_i(e); best.j = ev_j(e); }
            cands[w] = best;
        }
    }
}

template <bool XY_SMEM>
__device__ __forceinline__ float2 ldp(const float2 *s_p, const float2 *__restrict__ g_p, int k)
{
    return XY_SMEM ? s_p[k] : g_p[k];
}

// Float pre-test of one window end, done before any double arithmetic.  The
// window has the pair's point A at one end and T at the other; at the
// pair's slope S its width is (T.y - A.y) - (T.x - A.x) S (a top end) or
// its negative (a bottom end).  With sf the float slope dy / dx, the float
// estimate v = fma(-(T.x - A.x), sf, T.y - A.y) is within about
// 2^-20.5 (|dY| + |dX| |S|) of that width, and the double width the sweep
// records (projections y - s x in double, then their difference) within
// 2^-49 (|T.y| + |A.y| + |S| (|T.x| + |A.x|)).  The slack below is at least
// twice their sum, so v - slack > wb (the lane's best width, rounded up)
// proves the window wider than the best: it cannot change the best and
// its double arithmetic (one division, three projections) is skipped.
// Sound for tame points (every operand a normal float, overflow to inf
// only ever disabling the test); the caller passes wb = +inf otherwise.
__device__ __forceinline__ bool f32_wider(float2 A, float2 T, float sf, bool top, float wb)
{
    const float dY = T.y - A.y, dX = T.x - A.x;
    float v = fmaf(-dX, sf, dY);
    if (!top) v = -v;
    const float slack = 0x1p-18f * (fabsf(T.y) + fabsf(A.y) + fabsf(sf) * (fabsf(T.x) + fabsf(A.x))) + 0x1p-100f;
    return v - slack > wb;
}

// One warp per sweeper, taking slope ranges from a shared counter.  The
// events of a range are applied 32 at a time, lane-parallel, with the
// conflict rule of the int16 sweep (an earlier swap next to this one, or at
// the far end of one of its windows, makes the lane wait for the next
// batch); a pair that is not adjacent is repaired by the whole warp.  Each
// swap scores its two windows, the float pre-test first.
template <bool XY_SMEM>
__global__ void __launch_bounds__(256) k_sweep_f32(const float2 *__restrict__ g_p, int n, int h,
                                                   const unsigned *__restrict__ ev,
                                                   const unsigned *__restrict__ range, int W,
                                                   const unsigned short *__restrict__ orders,
                                                   CandF *__restrict__ cands, int *__restrict__ meta,
                                                   const int *__restrict__ flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned *next_range = reinterpret_cast<unsigned *>(meta + 4);
    float2 *s_p = reinterpret_cast<float2 *>(smem);
    const size_t off0 = XY_SMEM ? (((size_t)n * 8 + 15) & ~(size_t)15) : 0;
    const size_t half = ((size_t)n * 2 + 15) & ~(size_t)15;
    unsigned short *order = reinterpret_cast<unsigned short *>(smem + off0 + warp * 2 * half);
    unsigned short *pos = reinterpret_cast<unsigned short *>(smem + off0 + warp * 2 * half + half);
    if (XY_SMEM) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_p[k] = g_p[k];
        __syncthreads();
    }
    const int g = blockIdx.x * nwarp + warp;   // this sweeping warp
    if (g >= W) return;                          // candidate slots exist for W warps
    const bool pretest = flags[1] != 0;
    // the residue test of the conflict check needs h - 1 >= 8 and n <= 3 (h - 1)
    const int H = h - 1;
    const bool fold_ok = H >= 8 && n <= 3 * H;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    auto PT = [&](int k) { return ldp<XY_SMEM>(s_p, g_p, k); };
    CandF best = candf_empty();
    float wb = INFINITY;   // the best width rounded up (>= 0), +inf while none or without the pre-test
    auto offer = [&](double wd, double t, double sl, int i, int j) {
        CandF c;
        c.w = wd; c.t = t; c.s = sl; c.i = i; c.j = j; c.valid = 1; c.pad = 0;
        if (candf_better(c, best)) {
            best = c;
            if (pretest) wb = fmaxf(__double2float_ru(wd), 0.f);
        }
    };
    // ranges are taken in slope order from a shared counter until none is left
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(next_range, 1u);
        w = __shfl_sync(FULL, w, 0);
        if (w >= (unsigned)W) break;
        const unsigned start = range[2 * w], end = range[2 * w + 1];
        if (start >= end) continue;
        __syncwarp();
        load_order(orders + (size_t)w * n, n, order, pos, lane);
        __syncwarp();
        unsigned k = start;
        // a window of 64 events: this batch's (e_cur) and the next one's
        unsigned e_cur = (k + lane < end) ? ev[k + lane] : 0u;
        unsigned e_nxt = (k + 32 + lane < end) ? ev[k + 32 + lane] : 0u;
        while (k < end) {
            const unsigned navail = min(32u, end - k);
            const bool valid = (unsigned)lane < navail;
            int a = ev_i(e_cur), b = ev_j(e_cur);
            float2 Pa = PT(a), Pb = PT(b);
            if (Pa.x > Pb.x) {
                const int t = a; a = b; b = t;
                const float2 tp = Pa; Pa = Pb; Pb = tp;
            }
            const int pa = valid ? pos[a] : 0, pb = valid ? pos[b] : 0;
            const bool done = valid && pb < pa;
            const bool simple = valid && !done && pb == pa + 1;
            const bool repair = valid && !done && !simple;
            bool conflict = false;
            if (fold_ok) {
                // two simple swaps at p and q conflict only if q - p is within 2
                // of 0 or of +-H, so p mod H and q mod H are within 2 of each
                // other, cyclically, and then share a cell of width 4 in one of
                // three grids (the last one shifted across the wrap); lanes that
                // share a cell are treated as conflicting (a superset)
                int f = pa;
                if (f >= H) f -= H;
                if (f >= H) f -= H;
                int f2 = f + 2;
                const unsigned none = 0x40000000u | (unsigned)lane;
                const unsigned cA = simple ? (unsigned)(f >> 2) : none;
                const unsigned cB = simple ? (unsigned)(f2 >> 2) : none;
                if (f2 >= H) f2 -= H;
                const unsigned cC = simple ? (unsigned)(f2 >> 2) : none;
                const unsigned nearm = __match_any_sync(FULL, cA) | __match_any_sync(FULL, cB) |
                                       __match_any_sync(FULL, cC);
                const unsigned simm = __ballot_sync(FULL, simple);
                conflict = simple && (nearm & simm & lanemask_lt) != 0u;
            } else {
                const unsigned me = simple ? (((unsigned)pa << 1) | 1u) : 0u;
                for (int t = 0; t < 31; ++t) {
                    const unsigned o = __shfl_sync(FULL, me, t);
                    if (!simple || t >= lane || !(o & 1u)) continue;
                    const int d = abs(pa - (int)(o >> 1));
                    if (d <= 2 || abs(d - H) <= 1) conflict = true;
                }
            }
            const unsigned bad = __ballot_sync(FULL, repair || conflict);
            const int cut = bad ? __ffs(bad) - 1 : (int)navail;
            int advance;
            if (cut > 0) {
                const bool go = simple && lane < cut;
                const int top = pa + h - 1, bot = pa - h + 2;
                const bool rt = go && top < n && top > pa + 1, rb = go && bot >= 0 && bot < pa;
                const int it = rt ? order[top] : 0, ib = rb ? order[bot] : 0;
                __syncwarp();
                if (go) {
                    order[pa] = (unsigned short)b;
                    order[pa + 1] = (unsigned short)a;
                    pos[b] = (unsigned short)pa;
                    pos[a] = (unsigned short)(pa + 1);
                }
                __syncwarp();
                if (go) {
                    const float2 Tt = PT(it), Tb = PT(ib);
                    const float sf = __fdividef(Pb.y - Pa.y, Pb.x - Pa.x);
                    const bool wt = top < n && !(rt && f32_wider(Pa, Tt, sf, true, wb));
                    const bool wbm = bot >= 0 && !(rb && f32_wider(Pa, Tb, sf, false, wb));
                    if (wt || wbm) {
                        const double sl = slope_of(Pa, Pb);
                        const double K = zf(Pa, sl);
                        const int i = min(a, b), j = max(a, b);
                        if (wt) {
                            const double kt = rt ? zf(Tt, sl) : K;
                            offer(kt - K, 0.5 * (K + kt), sl, i, j);
                        }
                        if (wbm) {
                            const double kb = rb ? zf(Tb, sl) : K;
                            offer(K - kb, 0.5 * (kb + K), sl, i, j);
                        }
                    }
                }
                advance = cut;
            } else {
                // lane 0's pair is not adjacent: every point between its two
                // points meets them at this slope (the order is sorted just
                // before it), so the block is put in the order just after the
                // slope, x descending (a stable sort: equal x never cross), and
                // every window with an end in the block is scored.  A block in
                // strictly ascending x (the usual case) is reversed by the warp.
                const int lo = __shfl_sync(FULL, pa, 0), hi = __shfl_sync(FULL, pb, 0);
                const int ra = __shfl_sync(FULL, a, 0), rb = __shfl_sync(FULL, b, 0);
                const double rsl = slope_of(PT(ra), PT(rb));
                bool asc = true;
                for (int u = lo + lane; u < hi; u += 32) asc = asc && PT(order[u]).x < PT(order[u + 1]).x;
                if (__all_sync(FULL, asc)) {
                    for (int u = lane; u < (hi - lo + 1) / 2; u += 32) {
                        const unsigned short ou = order[lo + u], ov = order[hi - u];
                        order[lo + u] = ov;
                        order[hi - u] = ou;
                    }
                } else if (lane == 0) {
                    for (int u = lo + 1; u <= hi; ++u) {
                        const unsigned short v = order[u];
                        const float xv = PT(v).x;
                        int t = u - 1;
                        while (t >= lo && PT(order[t]).x < xv) {
                            order[t + 1] = order[t];
                            --t;
                        }
                        order[t + 1] = v;
                    }
                }
                __syncwarp();
                for (int u = lo + lane; u <= hi; u += 32) pos[order[u]] = (unsigned short)u;
                __syncwarp();
                const int pi = min(ra, rb), pj = max(ra, rb);
                for (int q = lo + lane; q <= hi; q += 32) {
                    if (q + h - 1 < n) {
                        const double zb = zf(PT(order[q]), rsl), zt = zf(PT(order[q + h - 1]), rsl);
                        offer(zt - zb, 0.5 * (zb + zt), rsl, pi, pj);
                    }
                    if (q - h + 1 >= 0) {
                        const double zb = zf(PT(order[q - h + 1]), rsl), zt = zf(PT(order[q]), rsl);
                        offer(zt - zb, 0.5 * (zb + zt), rsl, pi, pj);
                    }
                }
                __syncwarp();
                advance = 1;
            }
            // slide the 64-event window by `advance`
            const int src = (lane + advance) & 31;
            const unsigned c1 = __shfl_sync(FULL, e_cur, src);
            const unsigned c2 = __shfl_sync(FULL, e_nxt, src);
            const bool from_cur = lane + advance < 32;
            k += advance;
            e_cur = from_cur ? c1 : c2;
            const unsigned q = k + 32 + lane;
            e_nxt = from_cur ? c2 : ((q < end) ? ev[q] : 0u);
        }
    }
    best = candf_warp_best(best);
    if (lane == 0) cands[W + g] = best;
}

__global__ void __launch_bounds__(1024) k_argmin_f32(const CandF *__restrict__ cands, int count,
                                                     const int *__restrict__ bad, lms_result *__restrict__ out)
{
    __shared__ CandF s_best[32];
    CandF best = candf_empty();
    for (int k = threadIdx.x; k < count; k += blockDim.x)
        if (candf_better(cands[k], best)) best = cands[k];
    best = candf_warp_best(best);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (warp != 0) return;
    best = lane < (int)(blockDim.x >> 5) ? s_best[lane] : candf_empty();
    best = candf_warp_best(best);
    if (lane != 0) return;
    lms_result r;
    r.w_num = r.w_den = r.s_num = r.s_den = r.t_num = r.t_den = 0;
    r.algorithm = LMS_ALGO_SWEEP;
    r.theta1 = best.s;
    r.theta2 = best.t;
    const double half = 0.5 * best.w;
    r.med_sq = half * half;
    r.i = best.i;
    r.j = best.j;
    r.status = *bad ? LMS_ERR_RANGE
                    : (!best.valid ? LMS_ERR_INTERNAL : (best.i < 0 ? LMS_ERR_VERTICAL : LMS_OK));
    *out = r;
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t sweep_f32_extra_bytes(int n, int W)
{
    int Pn = 1;
    while (Pn < n) Pn <<= 1;
    size_t b = a256(16);                                    // non-finite flag
    b += a256((size_t)n * 8);                               // float2 points
    b += a256((size_t)2 * W * sizeof(CandF));               // candidates
    if (n > SORT_SMEM_N) b += a256((size_t)W * Pn * 8) + a256((size_t)W * Pn * 2);
    return b;
}

// The float32 fit: the event pipeline with the double-slope key, the float
// sweep, and the final reduction.  `out` is the device result.
cudaError_t launch_sweep_f32_fit(const SweepPlan &p, const float *x, const float *y, void *fscratch,
                                 lms_result *out, cudaStream_t st)
{
    const int n = p.n;
    int Pn = 1;
    while (Pn < n) Pn <<= 1;
    unsigned char *q = static_cast<unsigned char *>(fscratch);
    int *bad = reinterpret_cast<int *>(q);
    q += a256(16);
    float2 *P = reinterpret_cast<float2 *>(q);
    q += a256((size_t)n * 8);
    CandF *cands = reinterpret_cast<CandF *>(q);
    q += a256((size_t)2 * p.W * sizeof(CandF));
    long long *gkeys = nullptr;
    unsigned short *gidx = nullptr;
    if (n > SORT_SMEM_N) {
        gkeys = reinterpret_cast<long long *>(q);
        q += a256((size_t)p.W * Pn * 8);
        gidx = reinterpret_cast<unsigned short *>(q);
    }
    { StageTimer _t(STAGE_PACK, st); k_pack_f32<<<1, 1024, 0, st>>>(x, y, n, P, bad); }
    cudaError_t e = launch_events_prepare<KeyF32>(p, P, st);
    if (e != cudaSuccess) return e;
    e = launch_events_finish<KeyF32>(p, P, nullptr, st, true);
    if (e != cudaSuccess) return e;
    const int Ps = Pn < 1024 ? 1024 : Pn;
    const size_t init_smem = (n <= SORT_SMEM_N) ? (size_t)Ps * 16 : 0;   // sort words + merge scratch
    cudaFuncSetAttribute(k_sweep_init_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)init_smem);
    {
        StageTimer _t(STAGE_INIT, st);
        k_sweep_init_f32<<<p.W, 1024, init_smem, st>>>(P, n, p.h, p.ev, p.range, p.W, p.meta, p.base, p.orders, gkeys,
                                                      gidx, cands);
    }
    const size_t per = 2 * (((size_t)n * 2 + 15) / 16 * 16);
    const bool xs = (size_t)n * 8 + per <= 227 * 1024 && n <= 8192;
    const size_t xyb = xs ? ((size_t)n * 8 + 15) / 16 * 16 : 0;
    int spb = (int)((227 * 1024 - xyb) / per);
    spb = spb < 1 ? 1 : (spb > 8 ? 8 : spb);
    const size_t sw_smem = xyb + per * spb;
    // persistent: at most one CTA per SM (the shared memory allows no more),
    // every warp taking ranges from the counter
    const int blocks = std::min((p.W + spb - 1) / spb, p.C);
    const int G = std::min(blocks * spb, p.W);
    if (xs) {
        cudaFuncSetAttribute(k_sweep_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        StageTimer _t(STAGE_SWEEP, st);
        k_sweep_f32<true><<<blocks, 32 * spb, sw_smem, st>>>(P, n, p.h, p.ev, p.range, p.W, p.orders, cands, p.meta,
                                                             bad);
    } else {
        cudaFuncSetAttribute(k_sweep_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        StageTimer _t(STAGE_SWEEP, st);
        k_sweep_f32<false><<<blocks, 32 * spb, sw_smem, st>>>(P, n, p.h, p.ev, p.range, p.W, p.orders, cands, p.meta,
                                                              bad);
    }
    {
        StageTimer _t(STAGE_ARGMIN, st);
        k_argmin_f32<<<1, 1024, 0, st>>>(cands, p.W + G, bad, out);
    }
    return cudaGetLastError();
}

}  // namespace lms
