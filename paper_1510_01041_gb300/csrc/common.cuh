// common.cuh -- device helpers shared by the LMS kernels (sm_103a).
//
// Exact integer formulation (Sec. 1 Eq. 1, Sec. 3.1): at a candidate slope
// s = dy/dx (dx > 0) the projection of point k scaled by dx is the exact
// integer key_k = y_k * dx - x_k * dy = dx * (y_k - s x_k).  For int16
// coordinates |key| <= 2^32, window widths w = key_top - key_bottom < 2^34,
// and every cross-multiplied comparison below stays under 2^51: int64 is
// exact throughout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lms.h"

namespace lms {

constexpr unsigned FULL = 0xffffffffu;

// One scored window at one slope.  dx == 0 marks "no candidate".
struct Cand {
    long long w;    // window width times dx
    long long t;    // key_bottom + key_top (window centre times 2 dx)
    int dy, dx;     // slope dy/dx, dx > 0 (not necessarily reduced)
    int i, j;       // index pair with that slope (i < j)
};
static_assert(sizeof(Cand) == 32, "Cand layout");

__host__ __device__ __forceinline__ Cand cand_empty()
{
    Cand c;
    c.w = 0; c.t = 0; c.dy = 0; c.dx = 0; c.i = -1; c.j = -1;
    return c;
}

// Lexicographic order on (w, theta1, theta2, i, j) as exact rationals.
__host__ __device__ __forceinline__ bool cand_better(const Cand &a, const Cand &b)
{
    if (a.dx == 0) return false;
    if (b.dx == 0) return true;
    long long l = a.w * (long long)b.dx, r = b.w * (long long)a.dx;
    if (l != r) return l < r;
    l = (long long)a.dy * b.dx;
    r = (long long)b.dy * a.dx;
    if (l != r) return l < r;
    l = a.t * (long long)b.dx;
    r = b.t * (long long)a.dx;
    if (l != r) return l < r;
    if (a.i != b.i) return a.i < b.i;
    return a.j < b.j;
}

__device__ __forceinline__ Cand cand_shfl_xor(const Cand &c, int m)
{
    Cand o;
    o.w = __shfl_xor_sync(FULL, c.w, m);
    o.t = __shfl_xor_sync(FULL, c.t, m);
    o.dy = __shfl_xor_sync(FULL, c.dy, m);
    o.dx = __shfl_xor_sync(FULL, c.dx, m);
    o.i = __shfl_xor_sync(FULL, c.i, m);
    o.j = __shfl_xor_sync(FULL, c.j, m);
    return o;
}

// Warp-wide best; every lane returns the same record.
__device__ __forceinline__ Cand warp_best(Cand c)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        Cand o = cand_shfl_xor(c, m);
        if (cand_better(o, c)) c = o;
    }
    return c;
}

// Points are staged as one 32-bit word: x in the low half, y in the high half.
__host__ __device__ __forceinline__ int pack_xy(int x, int y)
{
    return (int)(((unsigned)y << 16) | ((unsigned)x & 0xffffu));
}
__device__ __forceinline__ int px(int p) { return (int)(short)(p & 0xffff); }
__device__ __forceinline__ int py(int p) { return p >> 16; }

// Scaled projection key_k at slope dy/dx.
__device__ __forceinline__ long long proj(int p, int dy, int dx)
{
    return (long long)py(p) * dx - (long long)px(p) * dy;
}

// Slope of the pair (p, q) with dx > 0; returns false when x_p == x_q.
__device__ __forceinline__ bool pair_slope(int p, int q, int &dy, int &dx)
{
    dx = px(q) - px(p);
    dy = py(q) - py(p);
    if (dx == 0) return false;
    if (dx < 0) { dx = -dx; dy = -dy; }
    return true;
}

// Exact, strictly order-preserving integer key of a slope dy/dx
// (|dy| < 2^16, 0 < dx < 2^16): floor(dy * 2^32 / dx).  Two different
// slopes differ by at least 1/(dx1 dx2) > 2^-32, so their keys differ;
// equal slopes give equal keys.  The quotient is assembled from three
// 16-bit digits, each estimated with a float reciprocal and corrected once
// with an exact integer remainder.
__device__ __forceinline__ long long slope_key(int dy, int dx)
{
    const unsigned a = (unsigned)(dy < 0 ? -dy : dy);
    const unsigned d = (unsigned)dx;
    const float rd = __frcp_rn((float)d);
    unsigned q0 = __float2uint_rz((float)a * rd);
    long long r = (long long)a - (long long)q0 * d;
    if (r < 0) { --q0; r += d; } else if (r >= (long long)d) { ++q0; r -= d; }
    unsigned t = (unsigned)r << 16;
    unsigned q1 = __float2uint_rz((float)t * rd);
    r = (long long)t - (long long)q1 * d;
    if (r < 0) { --q1; r += d; } else if (r >= (long long)d) { ++q1; r -= d; }
    t = (unsigned)r << 16;
    unsigned q2 = __float2uint_rz((float)t * rd);
    r = (long long)t - (long long)q2 * d;
    if (r < 0) { --q2; r += d; } else if (r >= (long long)d) { ++q2; r -= d; }
    long long Q = ((long long)q0 << 32) | ((long long)q1 << 16) | (long long)q2;
    if (dy < 0) return -(Q + (r != 0));
    return Q;
}

// Events are stored as two 16-bit point indices.  The first event of a
// group of equal slopes stores (i, j) with i < j in (low, high); every
// further event of the same group stores them swapped, so the order of the
// two halves carries the "continues the previous group" bit.
__device__ __forceinline__ unsigned ev_pack(int i, int j, bool cont)
{
    return cont ? ((unsigned)i << 16) | (unsigned)j : ((unsigned)j << 16) | (unsigned)i;
}
__device__ __forceinline__ bool ev_cont(unsigned e) { return (e & 0xffffu) > (e >> 16); }
__device__ __forceinline__ int ev_i(unsigned e) { return (int)min(e & 0xffffu, e >> 16); }
__device__ __forceinline__ int ev_j(unsigned e) { return (int)max(e & 0xffffu, e >> 16); }

// Triangular decode of a pair index p in [0, n(n-1)/2) into i < j.
__device__ __forceinline__ void pair_decode(long long p, int &i, int &j)
{
    int jj = (int)((1.0f + sqrtf(8.0f * (float)p + 1.0f)) * 0.5f);
    while ((long long)jj * (jj - 1) / 2 > p) --jj;
    while ((long long)(jj + 1) * jj / 2 <= p) ++jj;
    j = jj;
    i = (int)(p - (long long)jj * (jj - 1) / 2);
}

// Ascending bitonic sort of P = IPT * blockDim.x words, held IPT per thread
// in v (thread t holds positions t IPT .. t IPT + IPT - 1).  A step whose
// partner position (position ^ j) lies in the same thread runs in registers,
// one whose partner lies in another lane of the warp runs by shuffles, and
// only steps across warps pass through the shared scratch s (P words).  For
// the pair at positions i < i ^ j of merge size k the smaller value goes to
// i when i & k == 0 and to i ^ j otherwise.  Every thread of the CTA calls
// it; s may be reused once it returns.
template <int IPT, class T>
__device__ __forceinline__ void cta_sort_blocked(T (&v)[IPT], T *s, int P)
{
    const int t = threadIdx.x, lane = t & 31;
    const int base = t * IPT;
    for (int k = 2; k <= P; k <<= 1) {
        int j = k >> 1;
        if (j >= 32 * IPT) {
#pragma unroll
            for (int r = 0; r < IPT; ++r) s[base + r] = v[r];
            __syncthreads();
            for (; j >= 32 * IPT; j >>= 1) {
                for (int q = t; q < P / 2; q += blockDim.x) {
                    const int i = 2 * q - (q & (j - 1)), l = i + j;
                    const bool up = (i & k) == 0;
                    const T a = s[i], b = s[l];
                    if ((a > b) == up) { s[i] = b; s[l] = a; }
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < IPT; ++r) v[r] = s[base + r];
            __syncthreads();
        }
        for (; j >= IPT; j >>= 1) {
            const int m = j / IPT;
            const bool lower = (lane & m) == 0;
#pragma unroll
            for (int r = 0; r < IPT; ++r) {
                const T o = __shfl_xor_sync(FULL, v[r], m);
                const bool up = ((base + r) & k) == 0;
                v[r] = (lower == up) ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
            }
        }
#pragma unroll
        for (int jj = IPT / 2; jj >= 1; jj >>= 1) {
            if (jj < k) {
#pragma unroll
                for (int r = 0; r < IPT; ++r) {
                    if ((r & jj) == 0) {
                        const bool up = ((base + r) & k) == 0;
                        const T a = v[r], b = v[r ^ jj];
                        if ((a > b) == up) { v[r] = b; v[r ^ jj] = a; }
                    }
                }
            }
        }
    }
}

// Shared-memory slot of word p of an intermediate merge level: inside every
// aligned 128-byte row (R words) the word index is XORed with the row index
// mod R.  A thread stores IPT consecutive words, so plain slots put the
// threads of a warp that are R / IPT apart on one bank (16-way for 8-byte
// words and IPT = 8); with the XOR every bank takes the minimum two (8-byte)
// or one (4-byte) accesses of a warp store for IPT = 1 .. 16, and the merge
// reads of neighbouring threads spread the same way.  A permutation inside
// each row, so the arrays keep their size (P must be a multiple of R).
template <class T>
__device__ __forceinline__ int merge_slot(int p)
{
    constexpr int R = 128 / (int)sizeof(T);
    return p ^ ((p / R) & (R - 1));
}

// Ascending bitonic sort of the 32 IPT words a warp holds, IPT per lane in
// v (lane l holds positions l IPT .. l IPT + IPT - 1).  For the pair at
// positions i < i ^ j of merge size k the smaller value goes to i when
// i & k == 0; with positions counted inside the warp every run of the last
// merge (k = 32 IPT) is ascending.  Partners within a lane are compared in
// registers, partners in other lanes are exchanged by shuffles.
template <int IPT, class T>
__device__ __forceinline__ void warp_sort_blocked(T (&v)[IPT])
{
    const int lane = threadIdx.x & 31;
    const int base = lane * IPT;
#pragma unroll
    for (int k = 2; k <= 32 * IPT; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j >= IPT; j >>= 1) {
            const int m = j / IPT;
            const bool lower = (lane & m) == 0;
#pragma unroll
            for (int r = 0; r < IPT; ++r) {
                const T o = __shfl_xor_sync(FULL, v[r], m);
                const bool up = ((base + r) & k) == 0;
                v[r] = (lower == up) ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
            }
        }
#pragma unroll
        for (int j = (k >> 1) < IPT ? (k >> 1) : IPT / 2; j >= 1; j >>= 1) {
#pragma unroll
            for (int r = 0; r < IPT; ++r) {
                const int q = r ^ j;
                if (q > r) {
                    const bool up = ((base + r) & k) == 0;
                    const T a = v[r], b = v[q];
                    if ((a > b) == up) { v[r] = b; v[q] = a; }
                }
            }
        }
    }
}

// Ascending merge sort of P = IPT * blockDim.x words held IPT per thread in
// v (thread t holds positions t IPT ..), result in s (plain order); s2 is
// scratch of P words.  Each warp sorts its 32 IPT words in registers
// (warp_sort_blocked), then runs of width w = 32 IPT, 64 IPT, .. are merged
// pairwise: thread t produces the IPT outputs starting at t IPT of its
// merged run, finding its start on the merge path by a binary search (the
// diagonal split with A[i - 1] <= B[d - i], ties taken from the left run)
// and merging sequentially with the heads of both runs in registers.
// Intermediate levels use the slots of merge_slot; the last level writes
// plain positions.  Every thread of the CTA calls it.
template <int IPT, class T>
__device__ __forceinline__ void cta_merge_sort(T (&v)[IPT], T *s, T *s2, int P)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "merge_slot assumes 4- or 8-byte words");
    warp_sort_blocked<IPT>(v);
    const int t = threadIdx.x;
    const int o = t * IPT;
    // the number of merge levels decides where the first write goes so that
    // the last one lands in s
    int levels = 0;
    for (int w = 32 * IPT; w < P; w <<= 1) ++levels;
    const bool swz = P % (128 / (int)sizeof(T)) == 0;   // whole rows: the slots are a permutation
    auto slot = [&](int p) { return swz ? merge_slot<T>(p) : p; };
    T *src = (levels & 1) ? s2 : s, *dst = (levels & 1) ? s : s2;
#pragma unroll
    for (int r = 0; r < IPT; ++r) src[levels ? slot(o + r) : o + r] = v[r];
    __syncthreads();
    for (int w = 32 * IPT; w < P; w <<= 1) {
        const bool last = 2 * w >= P;
        const int base = o & ~(2 * w - 1);       // start of this thread's merged run
        const int d = o - base;                   // output offset inside it
        const int ba = base, bb = base + w;       // the two runs
        int lo = d > w ? d - w : 0, hi = d < w ? d : w;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (src[slot(ba + m)] <= src[slot(bb + d - 1 - m)]) lo = m + 1; else hi = m;
        }
        int ia = lo, ib = d - lo;
        T a = src[slot(ba + (ia < w ? ia : w - 1))];
        T b = src[slot(bb + (ib < w ? ib : w - 1))];
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            // branch-free: the taken head is replaced by the next word of its
            // run (one load, skipped past the run's end)
            const bool take_a = ib >= w || (ia < w && a <= b);
            const T x = take_a ? a : b;
            v[r] = x;
            ia += take_a;
            ib += !take_a;
            const int nx = take_a ? ba + ia : bb + ib;
            const T y = (take_a ? ia : ib) < w ? src[slot(nx)] : x;
            a = take_a ? y : a;
            b = take_a ? b : y;
        }
#pragma unroll
        for (int r = 0; r < IPT; ++r) dst[last ? o + r : slot(o + r)] = v[r];
        __syncthreads();
        T *tmp = src; src = dst; dst = tmp;
    }
}

// Fills P = IPT * blockDim.x words with fill(position) and merge-sorts them
// into s (s2: scratch of P words).
template <int IPT, class T, class F>
__device__ __forceinline__ void cta_fill_merge_sort(T *s, T *s2, int P, F fill)
{
    // which thread starts with which value does not matter to a sort: read
    // the inputs with consecutive threads on consecutive positions
    T v[IPT];
#pragma unroll
    for (int r = 0; r < IPT; ++r) v[r] = fill(r * (int)blockDim.x + (int)threadIdx.x);
    cta_merge_sort<IPT>(v, s, s2, P);
}

// The same for P / blockDim.x in {1, 2, 4, 8, 16}; false (nothing done)
// for other sizes.
template <class T, class F>
__device__ bool cta_fill_merge_sort_any(T *s, T *s2, int P, F fill)
{
    switch (P / (int)blockDim.x) {
        case 1: cta_fill_merge_sort<1>(s, s2, P, fill); return true;
        case 2: cta_fill_merge_sort<2>(s, s2, P, fill); return true;
        case 4: cta_fill_merge_sort<4>(s, s2, P, fill); return true;
        case 8: cta_fill_merge_sort<8>(s, s2, P, fill); return true;
        case 16: cta_fill_merge_sort<16>(s, s2, P, fill); return true;
        default: return false;
    }
}

// Merge of the sorted runs a[0, len) and b[0, len) (global memory) into
// out[0, 2 len) through shared memory s of 2 TILE words: the outputs are cut
// into tiles of TILE; the merge-path splits at every tile boundary (the
// number of a's words among the first d outputs, ties taken from a first)
// are found first, one binary search per boundary, all at once; then each
// tile's inputs (TILE words of the two runs together) are read with
// coalesced loads into s, merged there (each thread finds its start on the
// tile's merge path by a binary search and merges its share into the second
// half of s) and written out with coalesced stores.  Global memory is only
// streamed, never chased word by word.  Every thread of the CTA calls it.
constexpr int MERGE_SPLITS_MAX = 64;
template <int TILE, class T>
__device__ void cta_merge_tiled(const T *a, const T *b, int len, T *out, T *s)
{
    __shared__ int s_split[MERGE_SPLITS_MAX + 1];
    const int total = 2 * len;
    for (int t0 = 0; t0 < total; t0 += TILE * MERGE_SPLITS_MAX) {
        const int nt = min(MERGE_SPLITS_MAX, (total - t0 + TILE - 1) / TILE);
        for (int t = threadIdx.x; t <= nt; t += blockDim.x) {
            const int d = min(t0 + t * TILE, total);
            int lo = d > len ? d - len : 0, hi = d < len ? d : len;
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if (a[m] <= b[d - 1 - m]) lo = m + 1; else hi = m;
            }
            s_split[t] = lo;
        }
        __syncthreads();
        for (int t = 0; t < nt; ++t) {
            const int d0 = t0 + t * TILE, d1 = min(d0 + TILE, total);
            const int i0 = s_split[t], i1 = s_split[t + 1];
            const int j0 = d0 - i0, j1 = d1 - i1;
            const int na = i1 - i0, nb = j1 - j0, m = d1 - d0;
            for (int k = threadIdx.x; k < na; k += blockDim.x) s[k] = a[i0 + k];
            for (int k = threadIdx.x; k < nb; k += blockDim.x) s[na + k] = b[j0 + k];
            __syncthreads();
            const int per = (m + (int)blockDim.x - 1) / (int)blockDim.x;
            const int dd = (int)threadIdx.x * per;
            if (dd < m) {
                int lo = dd > nb ? dd - nb : 0, hi = dd < na ? dd : na;
                while (lo < hi) {
                    const int mm = (lo + hi) >> 1;
                    if (s[mm] <= s[na + dd - 1 - mm]) lo = mm + 1; else hi = mm;
                }
                int i = lo, j = dd - lo;
                for (int o = dd; o < dd + per && o < m; ++o) {
                    const bool take_a = j >= nb || (i < na && s[i] <= s[na + j]);
                    s[TILE + o] = take_a ? s[i++] : s[na + j++];
                }
            }
            __syncthreads();
            for (int k = threadIdx.x; k < m; k += blockDim.x) out[d0 + k] = s[TILE + k];
            __syncthreads();
        }
    }
}

// Ascending sort of the P words key(0 .. P - 1) (P a power of two, a
// multiple of Q) into global memory: chunks of Q words (Q = IPT blockDim.x
// with IPT in 1 .. 16) are merge-sorted in shared memory (s: 2 Q words)
// and written to A, then runs are merged pairwise between A and B
// (cta_merge_tiled, with s as its tile space).  Returns the buffer holding
// the result.  Every thread of the CTA calls it.
template <int Q, class T, class F>
__device__ T *cta_sort_chunked(T *s, T *A, T *B, int P, F key)
{
    for (int c = 0; c < P; c += Q) {
        cta_fill_merge_sort_any(s, s + Q, Q, [&](int k) { return key(c + k); });
        for (int k = threadIdx.x; k < Q; k += blockDim.x) A[c + k] = s[k];
        __syncthreads();
    }
    T *src = A, *dst = B;
    for (int len = Q; len < P; len <<= 1) {
        for (int r = 0; r < P; r += 2 * len) cta_merge_tiled<Q>(src + r, src + r + len, len, dst + r, s);
        __syncthreads();
        T *t = src; src = dst; dst = t;
    }
    return src;
}

// Fills P = IPT * blockDim.x words with fill(position), sorts them and
// leaves the ascending result in s.
template <int IPT, class T, class F>
__device__ __forceinline__ void cta_fill_sort(T *s, int P, F fill)
{
    // inputs read by consecutive threads at consecutive positions (the
    // starting arrangement of a sort is arbitrary)
    T v[IPT];
    const int base = threadIdx.x * IPT;
#pragma unroll
    for (int r = 0; r < IPT; ++r) v[r] = fill(r * (int)blockDim.x + (int)threadIdx.x);
    cta_sort_blocked<IPT>(v, s, P);
#pragma unroll
    for (int r = 0; r < IPT; ++r) s[base + r] = v[r];
    __syncthreads();
}

// The same for P / blockDim.x in {1, 2, 4, 8, 16} (P a power of two, at least
// blockDim.x); returns false (nothing done) for other sizes.
template <class T, class F>
__device__ bool cta_fill_sort_any(T *s, int P, F fill)
{
    switch (P / (int)blockDim.x) {
        case 1: cta_fill_sort<1>(s, P, fill); return true;
        case 2: cta_fill_sort<2>(s, P, fill); return true;
        case 4: cta_fill_sort<4>(s, P, fill); return true;
        case 8: cta_fill_sort<8>(s, P, fill); return true;
        case 16: cta_fill_sort<16>(s, P, fill); return true;
        default: return false;
    }
}

// A range's start order (global, written by the start sort) into the warp's
// order and position arrays.  When n is a multiple of 8 the order is read as
// 16-byte words, four per lane in flight (the slice starts at w n 2 bytes of
// a 256-byte aligned array, so it is 16-byte aligned), and stored to shared
// memory as 16-byte words; else one 16-bit entry at a time.
__device__ __forceinline__ void load_order(const unsigned short *__restrict__ src, int n, unsigned short *order,
                                           unsigned short *pos, int lane)
{
    if ((n & 7) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *o4 = reinterpret_cast<uint4 *>(order);
        const int n8 = n >> 3;
        for (int v0 = 0; v0 < n8; v0 += 4 * 32) {
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int v = v0 + u * 32 + lane;
                q[u] = v < n8 ? s4[v] : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int v = v0 + u * 32 + lane;
                if (v >= n8) continue;
                o4[v] = q[u];
                const unsigned wds[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    pos[wds[r] & 0xffffu] = (unsigned short)(8 * v + 2 * r);
                    pos[wds[r] >> 16] = (unsigned short)(8 * v + 2 * r + 1);
                }
            }
        }
    } else {
        for (int a = lane; a < n; a += 32) {
            const unsigned short p = src[a];
            order[a] = p;
            pos[p] = (unsigned short)a;
        }
    }
}

}  // namespace lms
