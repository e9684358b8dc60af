// sweep.cu -- exact kinetic sweep over the dual arrangement (sm_103a).
//
// Algorithm 1 (Sec. 3.4) sorts all n projections at every one of the
// n(n-1)/2 vertices.  Between two consecutive vertex slopes the sorted order
// of the projections z_k(s) = y_k - s x_k does not change, and at a vertex
// only the points that meet there swap (the vertical sweep of Souvaine and
// Steele cited in Sec. 2).  A window of h consecutive positions therefore
// changes its width function only when one of its two end positions changes
// occupant, so it is enough to (1) score every window once at the first
// vertex of a slope range and (2) at each later vertex re-score the windows
// with an end inside a swapped run (the equioscillation argument of
// Sec. 3.3: the optimal bracelet has a vertex at one end).
//
// Pipeline (all on one stream, no host synchronisation):
//   pack      points -> 32-bit words
//   sample    S pseudo-random pairs -> exact slope keys
//   sort      sample: shared-memory merge-sorted chunks, one rank merge
//   splitters quantiles of the sample -> slope-bucket boundaries (a key
//             that fills whole quantiles gets a bucket of its own)
//   count     every pair -> bucket, per-CTA shared-memory histograms (a
//             restricted pass instead lists the pairs of the kept buckets:
//             all-pairs tiles with a float cover test, or a band scan over
//             the points sorted at each cover's lower slope)
//   prefix    per-bucket offsets of each CTA; scan -> bucket starts
//   scatter   every pair -> its bucket (4-byte event)
//   segsort   each bucket sorted by exact slope key in shared memory (a
//             bucket above SEG_CAP events by one more level of sample sort
//             inside it); the event word records "same slope as previous"
//   plan      contiguous bucket ranges with equal event counts -> sweepers
//   init      per sweeper: sort the points at its first slope, score every
//             window there
//   sweep     per sweeper (one warp): apply the events in slope order,
//             re-score the touched windows, keep the best
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace lms {

namespace {

constexpr long long KEY_INF = 0x7fffffffffffffffLL;
constexpr int TILE = 64;          // pair tile edge of the count / scatter passes
constexpr int CNT_THREADS = 512;  // threads of a count / scatter CTA
constexpr int SORT_CHUNK = 1024;  // smallest sample (one CTA of the chunk sort)
#ifndef SWEEP_RANGE_FACTOR
#define SWEEP_RANGE_FACTOR 4
#endif
constexpr int RANGE_FACTOR = SWEEP_RANGE_FACTOR;   // slope ranges per sweeping warp (dynamic load balance)
constexpr long long MIN_RANGE_EVENTS = 512;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Number of boundaries <= key among bnd[0..P2) (bnd padded with KEY_INF, P2 a
// power of two strictly greater than the number of real boundaries).
__device__ __forceinline__ int bucket_of(const long long *bnd, int P2, long long key)
{
    int pos = 0;
    for (int step = P2 >> 1; step >= 1; step >>= 1)
        if (bnd[pos + step - 1] <= key) pos += step;
    return pos;
}

// Bucket of the pair (i, j), -1 when x_i == x_j.  int16 points: the exact
// key, searched.  float points: the exact key costs a double division, so
// the slope is first estimated in float, dy / dx with the differences and
// the quotient each rounded once (relative error below 2^-21), and widened
// by 2^-18 relative on both sides (__fdividef is within 2 ulp for divisors
// in [2^-126, 2^126]; the range checks keep every operand normal); the
// interval's two ends are mapped to the
// key space (the double bits of a float are a shift and a re-bias of its
// own).  When both ends fall in one bucket the exact key does too; otherwise
// (about one pair in a few hundred), and wherever a float leaves the normal
// range, the exact key decides.
template <class G>
__device__ __forceinline__ int pair_bucket(const void *pts, int i, int j, const long long *s_bnd, int P2)
{
    if constexpr (std::is_same<G, KeyF32>::value) {
        const float2 *P = static_cast<const float2 *>(pts);
        const float2 a = P[i], c = P[j];
        if (a.x == c.x) return -1;
        if (a.y == c.y) return bucket_of(s_bnd, P2, 0);   // slope 0: key 0 exactly
        float dx = c.x - a.x, dy = c.y - a.y;
        if (dx < 0.f) { dx = -dx; dy = -dy; }
        const float q = __fdividef(dy, dx);
        const float aq = fabsf(q);
        if (dx >= 0x1p-100f && dx <= 0x1p100f && fabsf(dy) >= 0x1p-100f && aq >= 0x1p-100f && aq <= 0x1p100f) {
            // float -> key of the same value as a double
            auto fkey = [](float f) {
                const unsigned u = __float_as_uint(f);
                const long long mag = ((long long)(u & 0x7fffffffu) << 29) + (896LL << 52);
                return (u >> 31) ? ~mag : mag;
            };
            const float q0 = q * (1.f - 0x1p-18f), q1 = q * (1.f + 0x1p-18f);
            const long long klo = fkey(fminf(q0, q1)), khi = fkey(fmaxf(q0, q1));
            const int b = bucket_of(s_bnd, P2, klo);
            if (khi < s_bnd[b]) return b;
        }
    }
    long long key;
    if (!G::key(pts, i, j, key)) return -1;
    return bucket_of(s_bnd, P2, key);
}

// Upper-triangle tile decode: tile q -> (bi <= bj).
__device__ __forceinline__ void tile_decode(int q, int &bi, int &bj)
{
    int j = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while (j * (j + 1) / 2 > q) --j;
    while ((j + 1) * (j + 2) / 2 <= q) ++j;
    bj = j;
    bi = q - j * (j + 1) / 2;
}

// ---------------------------------------------------------------- pack
__global__ void k_pack(const short *__restrict__ x, const short *__restrict__ y, int n, int *__restrict__ xy)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        xy[k] = pack_xy(x[k], y[k]);
}

// ---------------------------------------------------------------- sample
template <class G>
__global__ void k_sample(const void *__restrict__ pts, int n, long long npairs, int S, long long *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const unsigned long long r = mix64(0x5851F42D4C957F2Dull + (unsigned long long)k * 0x9E3779B97F4A7C15ull);
    const long long p = (long long)__umul64hi(r, (unsigned long long)npairs);
    int i, j;
    pair_decode(p, i, j);
    long long key;
    out[k] = G::key(pts, i, j, key) ? key : KEY_INF;
}

// The sample (S keys, a power of two) is sorted in chunks of up to
// SAMPLE_CH keys, one CTA each, by the shared-memory merge sort, then the
// chunks are merged in one pass by ranking.
constexpr int SAMPLE_CH = 8192;

__global__ void __launch_bounds__(1024) k_sort_chunks(long long *__restrict__ keys, int S)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s = reinterpret_cast<long long *>(smem);
    const int P = S < SAMPLE_CH ? S : SAMPLE_CH;
    long long *g = keys + (size_t)blockIdx.x * P;
    cta_fill_merge_sort_any(s, s + P, P, [&](int k) { return g[k]; });
    for (int k = threadIdx.x; k < P; k += blockDim.x) g[k] = s[k];
}

// Merge of the S / SAMPLE_CH sorted chunks (at most 16) by ranking: the key
// at position p of chunk c goes to p plus the number of keys <= it in the
// chunks before c and < it in the chunks after (a stable order, every
// position taken once).  The binary searches over the chunks are
// independent and run together.
__global__ void __launch_bounds__(256) k_merge_chunks(const long long *__restrict__ src, long long *__restrict__ dst,
                                                      int S)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const int nch = S / SAMPLE_CH, c = k / SAMPLE_CH;
    const long long v = src[k];
    int r = k - c * SAMPLE_CH;
#pragma unroll
    for (int c2 = 0; c2 < 16; ++c2) {
        if (c2 >= nch || c2 == c) continue;
        const long long *o = src + (size_t)c2 * SAMPLE_CH;
        int pos = 0;
        if (c2 < c) {
#pragma unroll
            for (int step = SAMPLE_CH / 2; step >= 1; step >>= 1)
                if (o[pos + step - 1] <= v) pos += step;
            pos += o[pos] <= v;   // the loop leaves the last key untested
        } else {
#pragma unroll
            for (int step = SAMPLE_CH / 2; step >= 1; step >>= 1)
                if (o[pos + step - 1] < v) pos += step;
            pos += o[pos] < v;
        }
        r += pos;
    }
    dst[r] = v;
}

// ---------------------------------------------------------------- splitters
// Quantiles of the sorted sample become boundaries; a value that spans two
// or more quantile positions is a heavy slope and gets the singleton bucket
// [v, v + 1).  Boundaries are strictly increasing; the array is padded with
// KEY_INF to the power of two P2 > nbnd.
// bcount (optional): the number of keys the buckets will hold; then B is
// lowered to about *bcount / bper buckets.
__global__ void __launch_bounds__(1024) k_splitters(const long long *__restrict__ sorted, int S, int B,
                                                    long long *__restrict__ bnd, int *__restrict__ meta,
                                                    const int *__restrict__ bcount = nullptr, int bper = 1)
{
    extern __shared__ long long s_q[];   // the B - 1 quantiles (at most BND_MAX / 2)
    __shared__ int s_m;
    __shared__ int s_scan[1024];
    if (bcount) {
        const long long want = ((long long)max(*bcount, 0) + bper - 1) / bper;
        B = (int)min((long long)B, max(want, 1LL));
    }
    if (threadIdx.x < 32) {
        // first KEY_INF (invalid samples sort last), by a 32-way search
        const int lane = threadIdx.x;
        int lo = 0, hi = S;
        while (hi - lo > 32) {
            const int step = (hi - lo + 31) / 32;
            const int at = lo + (lane + 1) * step - 1;
            const int c = __popc(__ballot_sync(FULL, at < hi && sorted[at] < KEY_INF));
            lo += c * step;
            hi = min(hi, lo + step);
        }
        const int c = __popc(__ballot_sync(FULL, lo + lane < hi && sorted[lo + lane] < KEY_INF));
        if (lane == 0) s_m = lo + c;
    }
    __syncthreads();
    const int m = s_m;
    const int nq = (m > 0) ? B - 1 : 0;          // quantiles b = 1 .. B-1
    // the quantiles, read once with consecutive threads on consecutive b
    for (int b = 1 + threadIdx.x; b <= nq; b += blockDim.x) s_q[b - 1] = sorted[(long long)b * m / B];
    __syncthreads();
    const int per = (nq + blockDim.x - 1) / blockDim.x;
    const int b0 = 1 + threadIdx.x * per;
    auto q = [&](int b) { return s_q[b - 1]; };
    int cnt = 0;
    for (int b = b0; b < b0 + per && b <= nq; ++b) {
        const long long v = q(b);
        const bool first = (b == 1) || q(b - 1) != v;
        const bool last = (b == nq) || q(b + 1) != v;
        const bool heavy = !(first && last);
        if (first) ++cnt;
        if (heavy && last && (b == nq || q(b + 1) != v + 1)) ++cnt;
    }
    s_scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int v = (threadIdx.x >= (unsigned)off) ? s_scan[threadIdx.x - off] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    int o = s_scan[threadIdx.x] - cnt;
    for (int b = b0; b < b0 + per && b <= nq; ++b) {
        const long long v = q(b);
        const bool first = (b == 1) || q(b - 1) != v;
        const bool last = (b == nq) || q(b + 1) != v;
        const bool heavy = !(first && last);
        if (first) bnd[o++] = v;
        if (heavy && last && (b == nq || q(b + 1) != v + 1)) bnd[o++] = v + 1;
    }
    __syncthreads();
    const int nbnd = s_scan[blockDim.x - 1];
    int P2 = 1;
    while (P2 <= nbnd) P2 <<= 1;
    for (int k = nbnd + threadIdx.x; k < P2; k += blockDim.x) bnd[k] = KEY_INF;
    if (threadIdx.x == 0) {
        meta[0] = nbnd; meta[1] = P2; meta[2] = 0; meta[3] = 0; meta[5] = 0; meta[6] = 0;
        meta[7] = 0;   // events covered by the sweep's ranges (start sorts and k_sweep add to it)
        meta[10] = m;  // valid sampled keys
    }
}

// ---------------------------------------------------------------- count / scatter
// Both passes walk the same upper-triangle tiles in the same static order,
// so the scatter's per-CTA bucket cursors match the counts exactly.  (A
// restricted fit lists its pairs with the band scan below; the scatter then
// places the list, k_scatter_list, whatever the order.)
template <bool SCATTER, class G>
__global__ void __launch_bounds__(CNT_THREADS) k_bucket_pairs(const void *__restrict__ pts, int n,
                                                              const long long *__restrict__ bnd,
                                                              const int *__restrict__ meta,
                                                              unsigned *__restrict__ hist,
                                                              const unsigned *__restrict__ base,
                                                              unsigned *__restrict__ ev,
                                                              const unsigned char *__restrict__ keep)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    const int nbnd = meta[0], P2 = meta[1], NB = nbnd + 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) s_bnd[k] = bnd[k];
    unsigned *my_hist = hist + (size_t)blockIdx.x * BND_MAX;
    for (int k = threadIdx.x; k < NB; k += blockDim.x)
        s_cnt[k] = SCATTER ? base[k] + my_hist[k] : 0u;
    __syncthreads();
    const int T = (n + TILE - 1) / TILE;
    const int ntiles = T * (T + 1) / 2;
    const int il = threadIdx.x & (TILE - 1);
    constexpr int JPT = TILE * TILE / CNT_THREADS;      // j values per thread
    const int jl0 = (threadIdx.x / TILE) * JPT;
    for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
        int bi, bj;
        tile_decode(q, bi, bj);
        const int i = bi * TILE + il;
        if (i >= n) continue;
#pragma unroll 4
        for (int jj = 0; jj < JPT; ++jj) {
            const int j = bj * TILE + jl0 + jj;
            if (j <= i || j >= n) continue;
            const int b = pair_bucket<G>(pts, i, j, s_bnd, P2);
            if (b < 0 || (keep && !keep[b])) continue;
            const unsigned slot = atomicAdd(&s_cnt[b], 1u);
            if (SCATTER) ev[slot] = ev_pack(i, j, false);
        }
    }
    if (!SCATTER) {
        __syncthreads();
        for (int k = threadIdx.x; k < NB; k += blockDim.x) my_hist[k] = s_cnt[k];
    }
}

// ---------------------------------------------------------------- restricted count (band scan)
// The pairs of a restricted pass are those whose exact slope key lies in a
// kept bucket; the kept buckets form at most PRE_MAX covers, cover c the key
// range [Klo_c, Khi_c).  A pair (a, b) with x_a < x_b and slope s has
//     Z_b - Z_a = (x_b - x_a) (s 2^32 - Klo),   Z = y 2^32 - x Klo,
// so a pair with key in [Klo, Khi) has 0 <= Z_b - Z_a < (x_b - x_a)(Khi - Klo)
// <= X (Khi - Klo), X the span of x.  With the points sorted by Z, every such
// pair lies within a band of D = X (Khi - Klo) of each other: scanning from
// every point forward over the points whose Z exceeds its own by at most D
// meets every pair of the cover exactly once (from the earlier of the two),
// so the pass lists the kept pairs in O(n log n + band pairs) instead of
// testing all n (n - 1) / 2.  Each pair met is resolved exactly (slope key,
// its cover, its bucket, the keep flag); a pair counts only in the scan of
// the cover its key lies in, so no pair is listed twice.  Covers whose keys
// reach |K| >= 2^46 (slopes steeper than 2^14, where Z would overflow) or are
// unbounded are scanned with an unbounded band: every pair, resolved the
// same way.

// Per cover, one CTA: the sorted words ((Z - Zmin) >> sh) << 16 | index,
// sh the smallest shift that keeps the span below 2^47, into words[c n ..],
// and the band in those units, (D >> sh) + 1 (truncation moves a difference
// by less than one unit), or -1 for an unused cover, into band[c].
// gscr: 2 P words per cover when n > 8192 (chunked sort), else unused.
__global__ void __launch_bounds__(1024) k_band_sort(const int *__restrict__ xy, int n,
                                                    const long long *__restrict__ cov,
                                                    unsigned long long *__restrict__ words,
                                                    long long *__restrict__ band,
                                                    unsigned long long *__restrict__ gscr)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_mn[32], s_mx[32];
    __shared__ int s_xl[32], s_xh[32];
    const int c = blockIdx.x;
    const long long Klo = cov[2 * c], Khi = cov[2 * c + 1];
    if (Klo >= Khi) {
        if (threadIdx.x == 0) band[c] = -1;
        return;
    }
    const long long G = 1LL << 46;
    const bool bounded = Klo > -G && Khi < G;
    const long long K = bounded ? Klo : 0;
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    int xl = INT_MAX, xh = INT_MIN;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int p = xy[k];
        const long long z = ((long long)py(p) << 32) - (long long)px(p) * K;
        mn = min(mn, z);
        mx = max(mx, z);
        xl = min(xl, px(p));
        xh = max(xh, px(p));
    }
    for (int s = 16; s >= 1; s >>= 1) {
        mn = min(mn, __shfl_xor_sync(FULL, mn, s));
        mx = max(mx, __shfl_xor_sync(FULL, mx, s));
        xl = min(xl, __shfl_xor_sync(FULL, xl, s));
        xh = max(xh, __shfl_xor_sync(FULL, xh, s));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; s_xl[warp] = xl; s_xh[warp] = xh; }
    __syncthreads();
    mn = s_mn[0]; mx = s_mx[0]; xl = s_xl[0]; xh = s_xh[0];
    for (int w = 1; w < nw; ++w) {
        mn = min(mn, s_mn[w]); mx = max(mx, s_mx[w]);
        xl = min(xl, s_xl[w]); xh = max(xh, s_xh[w]);
    }
    const unsigned long long span = (unsigned long long)(mx - mn);
    const int bits = span ? 64 - __clzll((long long)span) : 0;
    const int sh = bits > 47 ? bits - 47 : 0;
    int P = 1;
    while (P < n) P <<= 1;
    auto word = [&](int k) -> unsigned long long {
        if (k >= n) return ~0ull;
        const int p = xy[k];
        const long long z = ((long long)py(p) << 32) - (long long)px(p) * K;
        return (((unsigned long long)(z - mn) >> sh) << 16) | (unsigned long long)k;
    };
    unsigned long long *s = reinterpret_cast<unsigned long long *>(smem);
    const unsigned long long *sorted = s;
    if (P <= 8192) {
        const int Ps = P < (int)blockDim.x ? (int)blockDim.x : P;
        cta_fill_merge_sort_any(s, s + Ps, Ps, word);
    } else {
        unsigned long long *A = gscr + (size_t)c * 2 * P;
        sorted = cta_sort_chunked<8192>(s, A, A + P, P, word);
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) words[(size_t)c * n + k] = sorted[k];
    if (threadIdx.x == 0) {
        // X (Khi - Klo) < 2^16 2^47: no overflow
        band[c] = bounded ? (((long long)(xh - xl) * (Khi - Klo)) >> sh) + 1 : LLONG_MAX;
    }
}

// Restricted count by the band scan: item (c, p) is position p of cover c's
// sorted words; its lane finds where its band ends (a binary search on the
// truncated Z), the warp flattens its 32 bands into one list of pairs and
// walks it 32 pairs at a time (a long band, the dense points near the line,
// no longer holds the warp with one lane busy), pushing every pair onto the
// warp's stack, which is resolved 32 pairs at a time with all lanes busy
// (the exact key, bucket search, keep test, count and list are the costly
// part).  Counts go to this CTA's row of hist, the kept pairs to list
// (meta[6] counts them).
constexpr int BAND_THREADS = 1024;
constexpr int BAND_WARPS = BAND_THREADS / 32;
constexpr int BAND_STACK = 64;   // per warp: at most 31 left + 32 pushed

__global__ void __launch_bounds__(BAND_THREADS) k_band_pairs(const int *__restrict__ xy, int n,
                                                             const long long *__restrict__ bnd,
                                                             unsigned *__restrict__ hist,
                                                             const unsigned char *__restrict__ keep,
                                                             const long long *__restrict__ cov,
                                                             const unsigned long long *__restrict__ words,
                                                             const long long *__restrict__ band,
                                                             int *__restrict__ meta, unsigned *__restrict__ list)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    __shared__ unsigned long long s_stack[BAND_WARPS][BAND_STACK];
    __shared__ long long s_cov[2 * PRE_MAX], s_band[PRE_MAX];
    __shared__ float s_flo[PRE_MAX], s_fhi[PRE_MAX];
    if (threadIdx.x < 2 * PRE_MAX) s_cov[threadIdx.x] = cov[threadIdx.x];
    if (threadIdx.x < PRE_MAX) {
        // float slope bounds of the cover, widened by 2^-18 relative (a pair's
        // float test below errs by about 2^-23): used only by unbounded bands
        const int c = threadIdx.x;
        s_band[c] = band[c];
        const long long lo = cov[2 * c], hi = cov[2 * c + 1];
        const double dlo = (double)lo * 0x1p-32, dhi = (double)hi * 0x1p-32;
        s_flo[c] = lo <= -(1LL << 62) ? -INFINITY : __double2float_rd(dlo - (fabs(dlo) * 0x1p-18 + 0x1p-30));
        s_fhi[c] = hi >= (1LL << 62) ? INFINITY : __double2float_ru(dhi + (fabs(dhi) * 0x1p-18 + 0x1p-30));
    }
    const int P2 = meta[1], NB = meta[0] + 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) s_bnd[k] = bnd[k];
    for (int k = threadIdx.x; k < NB; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long *stk = s_stack[threadIdx.x >> 5];
    const unsigned below = (1u << lane) - 1u;
    int top = 0;   // warp-uniform stack height
    // exact resolution of one stacked pair per lane
    auto resolve = [&](unsigned long long e, bool have) {
        bool kept = false;
        unsigned pr = 0;
        if (have) {
            const int c = (int)(e >> 32);
            pr = (unsigned)e;
            long long key;
            if (KeyI16::key(xy, (int)(pr >> 16), (int)(pr & 0xffffu), key) && key >= s_cov[2 * c] &&
                key < s_cov[2 * c + 1]) {
                const int b = bucket_of(s_bnd, P2, key);
                if (!keep || keep[b]) {
                    atomicAdd(&s_cnt[b], 1u);
                    kept = true;
                }
            }
        }
        const unsigned m = __ballot_sync(FULL, kept);
        if (m) {
            unsigned at = 0;
            if (lane == 0) at = atomicAdd(reinterpret_cast<unsigned *>(meta + 6), (unsigned)__popc(m));
            at = __shfl_sync(FULL, at, 0) + __popc(m & below);
            if (kept) list[at] = pr;
        }
    };
    const long long items = (long long)PRE_MAX * n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // whole warps take consecutive items, so the loop below stays warp-uniform
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < items; base += stride) {
        const long long it = base + lane;
        const int c = (int)(min(it, items - 1) / n);
        const int p = (int)(min(it, items - 1) - (long long)c * n);
        const long long B = s_band[c];
        bool act = it < items && B >= 0;
        if (!__any_sync(FULL, act)) continue;
        const unsigned long long *w = words + (size_t)c * n;
        const unsigned long long wp = act ? w[p] : 0ull;
        const long long kp = (long long)(wp >> 16);
        // the band's end: the first later position whose key exceeds kp + B
        int end = p + 1;
        if (act) {
            int lo = p + 1, hi = n;
            if (B != LLONG_MAX) {
                while (lo < hi) {
                    const int md = (lo + hi) >> 1;
                    if ((long long)(w[md] >> 16) - kp <= B) lo = md + 1; else hi = md;
                }
            } else {
                lo = n;
            }
            end = lo;
        }
        // the warp's bands flattened into one list of pairs, 32 at a time:
        // pair t belongs to the lane whose prefix range holds t
        const int L = act ? end - p - 1 : 0;
        int incl = L;
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += o;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(FULL, incl, j + step - 1);
                if (v <= t) j += step;
            }
            j = min(j, 31);
            const int pj = __shfl_sync(FULL, p, j), cj = __shfl_sync(FULL, c, j);
            const int exj = __shfl_sync(FULL, incl - L, j);
            const unsigned ipj = (unsigned)(__shfl_sync(FULL, wp, j) & 0xffffu);
            bool cand = false;
            unsigned long long e = 0;
            if (t < total) {
                const unsigned long long wq = words[(size_t)cj * n + pj + 1 + (t - exj)];
                const unsigned iq = (unsigned)(wq & 0xffffu);
                const unsigned a = min(ipj, iq), b = max(ipj, iq);
                e = ((unsigned long long)cj << 32) | (a << 16) | b;
                cand = true;
                if (s_band[cj] == LLONG_MAX) {
                    // unbounded band: every later point, pre-tested in float
                    const int Pp = xy[ipj], Pq = xy[iq];
                    int dx = px(Pq) - px(Pp), dy = py(Pq) - py(Pp);
                    if (dx < 0) { dx = -dx; dy = -dy; }
                    cand = dx != 0 && s_flo[cj] * (float)dx <= (float)dy && (float)dy <= s_fhi[cj] * (float)dx;
                }
            }
            const unsigned m = __ballot_sync(FULL, cand);
            if (m) {
                if (cand) stk[top + __popc(m & below)] = e;
                top += __popc(m);
                if (top >= 32) {
                    __syncwarp();
                    top -= 32;
                    const unsigned long long se = stk[top + lane];
                    __syncwarp();
                    resolve(se, true);
                }
            }
        }
    }
    __syncwarp();
    if (top > 0) resolve(lane < top ? stk[lane] : 0ull, lane < top);
    __syncthreads();
    unsigned *my_hist = hist + (size_t)blockIdx.x * BND_MAX;
    for (int k = threadIdx.x; k < NB; k += blockDim.x) my_hist[k] = s_cnt[k];
}

// Restricted count over all pairs, for small sets (n <= TILE_COUNT_MAX_N),
// where one sort of the points per cover costs more than testing every
// pair: upper-triangle tiles of RC_TILE x RC_TILE pairs, each pair's slope
// tested in float against the covers (widened by 2^-18 relative; with
// dx > 0 the test lo dx <= dy <= hi dx needs no division, dx and dy exact,
// one rounding of 2^-24 per product), the survivors (about one pair in a
// hundred) pushed onto the warp's stack and resolved 32 at a time exactly
// (key, bucket, keep) like the band scan's.
constexpr int TILE_COUNT_MAX_N = 8192;
constexpr int RC_TILE = 128;   // pair tile edge

__global__ void __launch_bounds__(BAND_THREADS) k_tile_pairs(const int *__restrict__ xy, int n,
                                                             const long long *__restrict__ bnd,
                                                             unsigned *__restrict__ hist,
                                                             const unsigned char *__restrict__ keep,
                                                             const long long *__restrict__ cov,
                                                             int *__restrict__ meta, unsigned *__restrict__ list)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    __shared__ unsigned s_stack[BAND_WARPS][BAND_STACK];
    __shared__ float2 s_fc[2 * PRE_MAX];   // sorted float covers, then +inf (the search never reads past)
    if (threadIdx.x < 2 * PRE_MAX) {
        const int c = threadIdx.x;
        float2 f = make_float2(INFINITY, INFINITY);
        if (c < PRE_MAX && cov[2 * c] < cov[2 * c + 1]) {
            const long long lo = cov[2 * c], hi = cov[2 * c + 1];
            const double dlo = (double)lo * 0x1p-32, dhi = (double)hi * 0x1p-32;
            f.x = lo <= -(1LL << 62) ? -INFINITY : __double2float_rd(dlo - (fabs(dlo) * 0x1p-18 + 0x1p-30));
            f.y = hi >= (1LL << 62) ? INFINITY : __double2float_ru(dhi + (fabs(dhi) * 0x1p-18 + 0x1p-30));
        }
        s_fc[c] = f;
    }
    const int P2 = meta[1], NB = meta[0] + 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) s_bnd[k] = bnd[k];
    for (int k = threadIdx.x; k < NB; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();
    // hull of the covers: the first one's lower end to the last used one's upper end
    float2 ghull = make_float2(INFINITY, -INFINITY);
    for (int c = 0; c < PRE_MAX && s_fc[c].x < INFINITY; ++c) {
        ghull.x = fminf(ghull.x, s_fc[c].x);
        ghull.y = fmaxf(ghull.y, s_fc[c].y);
    }
    const int lane = threadIdx.x & 31;
    unsigned *stk = s_stack[threadIdx.x >> 5];
    const unsigned below = (1u << lane) - 1u;
    int top = 0;   // warp-uniform stack height
    auto resolve = [&](unsigned pr, bool have) {
        bool kept = false;
        if (have) {
            long long key;
            if (KeyI16::key(xy, (int)(pr >> 16), (int)(pr & 0xffffu), key)) {
                const int b = bucket_of(s_bnd, P2, key);
                if (!keep || keep[b]) {
                    atomicAdd(&s_cnt[b], 1u);
                    kept = true;
                }
            }
        }
        const unsigned m = __ballot_sync(FULL, kept);
        if (m) {
            unsigned at = 0;
            if (lane == 0) at = atomicAdd(reinterpret_cast<unsigned *>(meta + 6), (unsigned)__popc(m));
            at = __shfl_sync(FULL, at, 0) + __popc(m & below);
            if (kept) list[at] = pr;
        }
    };
    const int T = (n + RC_TILE - 1) / RC_TILE;
    const int ntiles = T * (T + 1) / 2;
    const int il = threadIdx.x & (RC_TILE - 1);
    constexpr int JPT = RC_TILE * RC_TILE / BAND_THREADS;
    const int jl0 = (threadIdx.x / RC_TILE) * JPT;
    for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
        int bi, bj;
        tile_decode(q, bi, bj);
        const int i = bi * RC_TILE + il;
        const bool row = i < n;
        const int Pi = row ? __ldg(xy + i) : 0;
#pragma unroll 4
        for (int jj = 0; jj < JPT; ++jj) {
            const int j = bj * RC_TILE + jl0 + jj;
            bool cand = false;
            if (row && j > i && j < n) {
                const int Pj = __ldg(xy + j);
                int dx = px(Pj) - px(Pi), dy = py(Pj) - py(Pi);
                if (dx != 0) {
                    if (dx < 0) { dx = -dx; dy = -dy; }
                    const float fx = (float)dx, fy = (float)dy;
                    // the hull of all covers first: nearly every pair falls outside it
                    if (ghull.x * fx <= fy && fy <= ghull.y * fx) {
                        int c = 0;
#pragma unroll
                        for (int step = PRE_MAX; step >= 1; step >>= 1)
                            if (s_fc[c + step - 1].x * fx <= fy) c += step;
                        cand = c > 0 && fy <= s_fc[c - 1].y * fx;
                    }
                }
            }
            const unsigned m = __ballot_sync(FULL, cand);
            if (m) {
                if (cand) stk[top + __popc(m & below)] = ((unsigned)i << 16) | (unsigned)j;
                top += __popc(m);
                if (top >= 32) {
                    __syncwarp();
                    top -= 32;
                    const unsigned pr = stk[top + lane];
                    __syncwarp();
                    resolve(pr, true);
                }
            }
        }
    }
    __syncwarp();
    if (top > 0) resolve(lane < top ? stk[lane] : 0u, lane < top);
    __syncthreads();
    unsigned *my_hist = hist + (size_t)blockIdx.x * BND_MAX;
    for (int k = threadIdx.x; k < NB; k += blockDim.x) my_hist[k] = s_cnt[k];
}

// Pairs with distinct x (the candidate slopes of the whole set) into
// meta[5]: all pairs less those within groups of equal x, counted by a
// histogram of x in shared memory, one half of the int16 range at a time.
__global__ void __launch_bounds__(1024) k_distinct_x_pairs(const int *__restrict__ xy, int n, int *__restrict__ meta)
{
    extern __shared__ unsigned s_h[];   // 32768 counters
    unsigned long long same = 0;
    for (int half = 0; half < 2; ++half) {
        for (int k = threadIdx.x; k < 32768; k += blockDim.x) s_h[k] = 0u;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int x = px(xy[k]) + 32768;
            if ((x >> 15) == half) atomicAdd(&s_h[x & 32767], 1u);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 32768; k += blockDim.x) {
            const unsigned long long v = s_h[k];
            same += v * (v - (v > 0)) / 2;
        }
        __syncthreads();
    }
    for (int s = 16; s >= 1; s >>= 1) same += __shfl_xor_sync(FULL, same, s);
    __shared__ unsigned long long s_same[32];
    if ((threadIdx.x & 31) == 0) s_same[threadIdx.x >> 5] = same;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_same[w];
        meta[5] = (int)((unsigned long long)n * (unsigned long long)(n - 1) / 2 - t);
    }
}

// The listed pairs to their buckets (the order inside a bucket is left to
// the bucket sort); cursor[b] starts at the bucket's first slot.  Each CTA
// takes a contiguous part of the list, counts it per bucket in shared
// memory, reserves one range per bucket with a single global atomic, then
// places its pairs (bucket indices recomputed from the exact keys).
template <class G>
__global__ void __launch_bounds__(CNT_THREADS) k_scatter_list(const void *__restrict__ pts,
                                                              const long long *__restrict__ bnd,
                                                              const int *__restrict__ meta,
                                                              const unsigned *__restrict__ list,
                                                              unsigned *__restrict__ cursor,
                                                              unsigned *__restrict__ ev,
                                                              const int *__restrict__ mlist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    const int P2 = meta[1], NB = meta[0] + 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) s_bnd[k] = bnd[k];
    for (int k = threadIdx.x; k < NB; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();
    const unsigned m = (unsigned)*mlist;
    const unsigned per = (m + gridDim.x - 1) / gridDim.x;
    const unsigned q0 = min(m, blockIdx.x * per), q1 = min(m, q0 + per);
    auto bucket = [&](unsigned pr, int &b) {
        b = pair_bucket<G>(pts, (int)(pr >> 16), (int)(pr & 0xffffu), s_bnd, P2);
        return b >= 0;
    };
    for (unsigned q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int b;
        if (bucket(list[q], b)) atomicAdd(&s_cnt[b], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NB; k += blockDim.x)
        if (s_cnt[k]) s_cnt[k] = atomicAdd(&cursor[k], s_cnt[k]);
    __syncthreads();
    for (unsigned q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const unsigned pr = list[q];
        int b;
        if (bucket(pr, b)) ev[atomicAdd(&s_cnt[b], 1u)] = ev_pack((int)(pr >> 16), (int)(pr & 0xffffu), false);
    }
}

// Resplit of a restricted pass: S keys of evenly spaced entries of the
// list of kept pairs (the list is in tile order, unrelated to the slopes).
template <class G>
__global__ void k_list_sample(const void *__restrict__ pts, const unsigned *__restrict__ list,
                              const int *__restrict__ mlist, int S, long long *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const unsigned m = (unsigned)max(*mlist, 0);
    long long k = KEY_INF;
    if (m > 0) {
        const unsigned pr = list[(unsigned)(((unsigned long long)s * m) / (unsigned)S)];
        if (!G::key(pts, (int)(pr >> 16), (int)(pr & 0xffffu), k)) k = KEY_INF;
    }
    out[s] = k;
}

// Resplit: bucket totals of the listed pairs (total zeroed by the caller).
template <class G>
__global__ void __launch_bounds__(CNT_THREADS) k_list_hist(const void *__restrict__ pts,
                                                           const long long *__restrict__ bnd,
                                                           const int *__restrict__ meta,
                                                           const unsigned *__restrict__ list,
                                                           const int *__restrict__ mlist,
                                                           unsigned *__restrict__ total)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    const int P2 = meta[1], NB = meta[0] + 1;
    for (int k = threadIdx.x; k < P2; k += blockDim.x) s_bnd[k] = bnd[k];
    for (int k = threadIdx.x; k < NB; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();
    const unsigned m = (unsigned)max(*mlist, 0);
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
        const unsigned pr = list[q];
        const int b = pair_bucket<G>(pts, (int)(pr >> 16), (int)(pr & 0xffffu), s_bnd, P2);
        if (b >= 0) atomicAdd(&s_cnt[b], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NB; k += blockDim.x)
        if (s_cnt[k]) atomicAdd(&total[k], s_cnt[k]);
}

// Per bucket: the number of valid sampled keys in it (the sample is sorted
// and the buckets are its quantile ranges, so two binary searches suffice).
__global__ void k_sample_counts(const long long *__restrict__ sorted, int S, const long long *__restrict__ bnd,
                                const int *__restrict__ meta, unsigned *__restrict__ counts)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int NB = meta[0] + 1;
    if (b >= NB) return;
    auto first_ge = [&](long long v) {
        int lo = 0, hi = S;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (sorted[m] < v) lo = m + 1; else hi = m; }
        return lo;
    };
    const int a = b == 0 ? 0 : first_ge(bnd[b - 1]);
    const int e = b == NB - 1 ? first_ge(KEY_INF) : first_ge(bnd[b]);
    counts[b] = (unsigned)(e - a);
}

// Per bucket: exclusive prefix over CTAs (in place) and the bucket total.
__global__ void k_bucket_prefix(unsigned *__restrict__ hist, int C, const int *__restrict__ meta,
                                unsigned *__restrict__ total)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > meta[0]) return;
    unsigned run = 0;
    for (int c = 0; c < C; ++c) {
        unsigned v = hist[(size_t)c * BND_MAX + b];
        hist[(size_t)c * BND_MAX + b] = run;
        run += v;
    }
    total[b] = run;
}

// Exclusive scan of bucket totals (in place, NB <= BND_MAX); base[NB] = E.
// copy (optional): receives the bucket starts too (the list scatter's cursors).
__global__ void __launch_bounds__(1024) k_bucket_scan(unsigned *__restrict__ base, const int *__restrict__ meta,
                                                      unsigned *__restrict__ copy = nullptr)
{
    __shared__ unsigned s[1024];
    const int NB = meta[0] + 1;
    const int per = (NB + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    unsigned sum = 0;
    for (int b = b0; b < b0 + per && b < NB; ++b) sum += base[b];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        unsigned v = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = s[threadIdx.x] - sum;
    for (int b = b0; b < b0 + per && b < NB; ++b) {
        unsigned v = base[b];
        base[b] = run;
        if (copy) copy[b] = run;
        run += v;
    }
    if (threadIdx.x == 1023) base[NB] = s[1023];
}

// ---------------------------------------------------------------- segsort
template <class G>
__device__ __forceinline__ long long event_key(const void *__restrict__ pts, unsigned e)
{
    long long k = KEY_INF;
    G::key(pts, ev_i(e), ev_j(e), k);
    return k;
}

__device__ __forceinline__ unsigned pair_of(unsigned e) { return ((unsigned)ev_i(e) << 16) | (unsigned)ev_j(e); }

// (slope key, index pair) order: inside a group of equal slopes the event
// with the smallest pair comes first.
__device__ __forceinline__ bool ev_less(long long ka, unsigned ea, long long kb, unsigned eb)
{
    return ka < kb || (ka == kb && pair_of(ea) < pair_of(eb));
}

// Merge of two sorted runs A, B of Hh words each (distinct words; B padded
// with ~0) into the first m outputs, written as events with the "same slope
// as the previous event" flag.  Every thread writes 16 consecutive outputs,
// its start on the merge path found by a binary search on its diagonal.
template <class Less, class Same>
__device__ void merge_halves_to_events(const unsigned long long *A, const unsigned long long *B, int Hh, int m,
                                       unsigned *__restrict__ out, Less less, Same same)
{
    const int d = (int)threadIdx.x * 16;
    if (d >= m) return;
    int lo = d > Hh ? d - Hh : 0, hi = d < Hh ? d : Hh;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (less(A[mid], B[d - 1 - mid])) lo = mid + 1; else hi = mid;
    }
    int i = lo, j = d - lo;
    unsigned long long prev = 0;
    bool have_prev = false;
    if (i > 0) { prev = A[i - 1]; have_prev = true; }
    if (j > 0 && (!have_prev || less(prev, B[j - 1]))) { prev = B[j - 1]; have_prev = true; }
    for (int o = d; o < d + 16 && o < m; ++o) {
        const bool take_a = j >= Hh || (i < Hh && less(A[i], B[j]));
        const unsigned long long v = take_a ? A[i++] : B[j++];
        const bool cont = have_prev && same(prev, v);
        out[o] = ev_pack((int)((v >> 16) & 0xffffu), (int)(v & 0xffffu), cont);
        prev = v;
        have_prev = true;
    }
}

// Sort of m <= SEG_CAP events src[0, m) whose keys lie in [klo, klo + span)
// into dst (src == dst allowed) by (exact slope key, pair), with the
// "same slope as the previous event" flags; false (dst untouched) when it
// cannot (a cell of equal shifted keys needing more than SEG_REPAIR_MAX
// passes, or no merge-sort shape for the size).  The word
// ((key - klo) >> sh) << 32 | pair, with sh the smallest shift that brings
// the span below 2^32, orders events by (key, pair) except inside a cell of
// equal shifted keys, where it orders them by pair alone.  The words are
// sorted in registers and shared memory; when sh > 0 the rare cells of two
// or more events are then put in (key, pair) order by odd-even
// transposition with the exact keys.  (int16 keys of one bucket span less
// than 2^32: sh = 0 and no repair.)  smem: SEG_CAP * 12 bytes.  Every
// thread of the CTA calls it.
template <class G>
__device__ bool sort_bucket_words(const void *__restrict__ xy, const unsigned *src, unsigned *dst, unsigned m,
                                  long long klo, unsigned long long span, unsigned char *smem)
{
    int P = 1;
    while (P < (int)m) P <<= 1;
    const int sh = span > 0xffffffffull ? 32 - __clzll((long long)span) : 0;
    unsigned long long *w = reinterpret_cast<unsigned long long *>(smem);
    auto word = [&](int k) {
        if (k >= (int)m) return ~0ull;
        const unsigned e = src[k];
        return (((unsigned long long)event_key<G>(xy, e) - (unsigned long long)klo) >> sh << 32) | pair_of(e);
    };
    auto exact = [&](unsigned long long v) {
        return event_key<G>(xy, ev_pack((int)((v >> 16) & 0xffffu), (int)(v & 0xffffu), false));
    };
    // (key, pair) order of two words; the padding word ~0 is last
    auto less = [&](unsigned long long u, unsigned long long v) {
        if (sh == 0 || (u >> 32) != (v >> 32) || u == ~0ull || v == ~0ull) return u < v;
        const long long ku = exact(u), kv = exact(v);
        return ku < kv || (ku == kv && (unsigned)u < (unsigned)v);
    };
    auto same = [&](unsigned long long u, unsigned long long v) {
        return (u >> 32) == (v >> 32) && (sh == 0 || exact(u) == exact(v));
    };
    auto repair = [&](unsigned long long *a, int len) {
        if (sh == 0) return true;
        int cells = 0;
        for (int k = threadIdx.x; k + 1 < len; k += blockDim.x) cells |= (a[k] >> 32) == (a[k + 1] >> 32);
        if (!__syncthreads_or(cells)) return true;
        for (int pass = 0; pass < SEG_REPAIR_MAX; ++pass) {
            int swapped = 0;
            for (int par = 0; par < 2; ++par) {
                for (int k = 2 * (int)threadIdx.x + par; k + 1 < len; k += 2 * (int)blockDim.x) {
                    const unsigned long long u = a[k], v = a[k + 1];
                    if ((u >> 32) == (v >> 32) && less(v, u)) {
                        a[k] = v;
                        a[k + 1] = u;
                        swapped = 1;
                    }
                }
                __syncthreads();
            }
            if (!__syncthreads_or(swapped)) return true;
        }
        return false;
    };
    __syncthreads();
    const int Pw = P < (int)blockDim.x ? (int)blockDim.x : P;
    if (2 * Pw > SEG_CAP * 3 / 2 && Pw == 2 * (int)blockDim.x * 8) {
        // too large for one merge sort and its scratch: two halves are
        // merge-sorted one after the other (scratch after both), then merged
        // by merge path straight into the event array
        const int Hh = Pw / 2;
        unsigned long long *A = w, *Bw = w + Hh, *scr = w + 2 * Hh;
        cta_fill_merge_sort<8>(A, scr, Hh, word);
        cta_fill_merge_sort<8>(Bw, scr, Hh, [&](int k) { return word(Hh + k); });
        __syncthreads();
        const bool ok = repair(A, Hh);
        if (!(ok && repair(Bw, (int)m - Hh))) return false;
        if (src == dst) __syncthreads();
        merge_halves_to_events(A, Bw, Hh, (int)m, dst, less, same);
        __syncthreads();
        return true;
    }
    // merge sort (registers, then merge-path levels) where its scratch copy
    // fits beside the words, else the register-blocked bitonic sort
    const bool sorted = 2 * Pw <= SEG_CAP * 3 / 2 ? cta_fill_merge_sort_any(w, w + Pw, Pw, word)
                                                   : cta_fill_sort_any(w, Pw, word);
    if (sorted) __syncthreads();
    if (!(sorted && repair(w, (int)m))) return false;
    for (int k = threadIdx.x; k < (int)m; k += blockDim.x) {
        const unsigned long long v = w[k];
        const bool cont = k > 0 && same(w[k - 1], v);
        dst[k] = ev_pack((int)((v >> 16) & 0xffffu), (int)(v & 0xffffu), cont);
    }
    __syncthreads();
    return true;
}

// Sort each bucket by (exact slope key, pair); buckets with more than
// SEG_CAP events are listed for k_segsort_big.  A bucket holding a single
// slope only needs its smallest pair moved to the front.
template <class G>
__global__ void __launch_bounds__(1024) k_segsort(const void *__restrict__ xy, unsigned *__restrict__ ev,
                                                  const unsigned *__restrict__ base,
                                                  const long long *__restrict__ bnd, int *__restrict__ meta,
                                                  int *__restrict__ oversize)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_key = reinterpret_cast<long long *>(smem);
    unsigned *s_ev = reinterpret_cast<unsigned *>(smem + SEG_CAP * sizeof(long long));
    __shared__ unsigned s_min[32];
    const int NB = meta[0] + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // The CTA's buckets are b = blockIdx.x + k gridDim.x.  Their sizes are read
    // all at once, 1024 at a time, and only the non-empty ones are visited:
    // walking them one by one costs a dependent global read per bucket, which
    // dominates when few buckets hold events (the branch-and-bound's kept
    // ones).
    __shared__ int s_list[1024];
    __shared__ int s_nl;
    for (long long c0 = blockIdx.x; c0 < NB; c0 += (long long)gridDim.x * blockDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) s_nl = 0;
        __syncthreads();
        {
            const long long bb = c0 + (long long)threadIdx.x * gridDim.x;
            if (bb < NB && base[bb + 1] > base[bb]) s_list[atomicAdd(&s_nl, 1)] = (int)bb;
        }
        __syncthreads();
        const int nl = s_nl;
        for (int q = 0; q < nl; ++q) {
            const int b = s_list[q];
            const unsigned off = base[b], m = base[b + 1] - off;
            const bool singleton = (b > 0 && b < NB - 1 && bnd[b] == bnd[b - 1] + 1);
            if (m == 1 || singleton) {
                // position of the smallest pair (pairs are distinct)
                unsigned best = 0xffffffffu, bpos = 0;
                for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
                    const unsigned pv = pair_of(ev[off + k]);
                    if (pv < best) { best = pv; bpos = k; }
                }
                for (int s = 16; s >= 1; s >>= 1) {
                    const unsigned ob = __shfl_xor_sync(FULL, best, s), op = __shfl_xor_sync(FULL, bpos, s);
                    if (ob < best) { best = ob; bpos = op; }
                }
                __syncthreads();
                if (lane == 0) { s_min[warp] = best; s_key[warp] = bpos; }
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned bb = 0xffffffffu, bp = 0;
                    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
                        if (s_min[q] < bb) { bb = s_min[q]; bp = (unsigned)s_key[q]; }
                    s_min[0] = bp;
                }
                __syncthreads();
                const unsigned mpos = s_min[0];
                const unsigned e0 = ev[off], em = ev[off + mpos];
                __syncthreads();
                for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
                    unsigned e = ev[off + k];
                    if (k == 0) e = em;
                    else if (k == mpos) e = e0;
                    ev[off + k] = ev_pack(ev_i(e), ev_j(e), k > 0);
                }
                continue;
            }
            if (m > (unsigned)SEG_CAP) {
                if (threadIdx.x == 0) {
                    const int slot = atomicAdd(&meta[2], 1);
                    oversize[slot] = b;
                }
                continue;
            }
            int P = 1;
            while (P < (int)m) P <<= 1;
            // an interior bucket: its keys lie in [bnd[b - 1], bnd[b])
            if (b > 0 && b < NB - 1 &&
                sort_bucket_words<G>(xy, ev + off, ev + off, m, bnd[b - 1],
                                     (unsigned long long)bnd[b] - (unsigned long long)bnd[b - 1], smem))
                continue;
            __syncthreads();
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                if (k < (int)m) {
                    const unsigned e = ev[off + k];
                    s_key[k] = event_key<G>(xy, e);
                    s_ev[k] = e;
                } else {
                    s_key[k] = KEY_INF;
                    s_ev[k] = 0xffffffffu;
                }
            }
            __syncthreads();
            for (int k = 2; k <= P; k <<= 1) {
                for (int j = k >> 1; j >= 1; j >>= 1) {
                    for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                        const int i = 2 * t - (t & (j - 1));
                        const int l = i + j;
                        const bool up = (i & k) == 0;
                        const long long a = s_key[i], c = s_key[l];
                        const unsigned ea = s_ev[i], ec = s_ev[l];
                        if (up ? ev_less(c, ec, a, ea) : ev_less(a, ea, c, ec)) {
                            s_key[i] = c; s_key[l] = a;
                            s_ev[i] = ec; s_ev[l] = ea;
                        }
                    }
                    __syncthreads();
                }
            }
            for (int k = threadIdx.x; k < (int)m; k += blockDim.x) {
                const unsigned e = s_ev[k];
                ev[off + k] = ev_pack(ev_i(e), ev_j(e), k > 0 && s_key[k] == s_key[k - 1]);
            }
        }
    }
}

// Buckets above SEG_CAP events, one CTA each, by one more level of sample
// sort inside the bucket: SB_SAMPLE evenly spaced events' keys are sorted
// and give F - 1 splitters (about SB_TARGET events a sub-bucket; a key equal
// to a splitter goes above it, so equal keys share a sub-bucket); one pass
// counts the events of every sub-bucket (and the bucket's least and largest
// key), a second moves them, grouped by sub-bucket, into the bucket's range
// of ev2, and each sub-bucket is then sorted from there into its place in ev
// by the word sort of the ordinary buckets, its keys in [splitter below,
// splitter above).  The buckets are sorted by (key, pair) and key ranges of
// sub-buckets do not overlap, so the result is the bucket's full sort.  A
// sub-bucket still above SEG_CAP (a slope shared by very many pairs) is
// sorted by the merge fallback: SEG_CAP-event chunks in shared memory, then
// pairwise merges with keys recomputed from the points.
constexpr int SB_SAMPLE = 2048;
constexpr int SB_TARGET = 6144;
constexpr int SB_MAX = 256;   // sub-buckets of one bucket

template <class G>
__device__ void sort_big_merge(const void *__restrict__ xy, unsigned *A, unsigned *scratch, unsigned m,
                               unsigned char *smem)
{
    long long *s_key = reinterpret_cast<long long *>(smem);
    unsigned *s_ev = reinterpret_cast<unsigned *>(smem + SEG_CAP * sizeof(long long));
    const int tid = threadIdx.x, nt = blockDim.x;
    // sorted runs of SEG_CAP events
    for (unsigned c0 = 0; c0 < m; c0 += SEG_CAP) {
        const int mc = (int)min((unsigned)SEG_CAP, m - c0);
        int P = 1;
        while (P < mc) P <<= 1;
        for (int k = tid; k < P; k += nt) {
            if (k < mc) {
                const unsigned e = A[c0 + k];
                s_key[k] = event_key<G>(xy, e);
                s_ev[k] = e;
            } else {
                s_key[k] = KEY_INF;
                s_ev[k] = 0xffffffffu;
            }
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j >= 1; j >>= 1) {
                for (int t = tid; t < P / 2; t += nt) {
                    const int i = 2 * t - (t & (j - 1));
                    const int l = i + j;
                    const bool up = (i & k) == 0;
                    const long long a = s_key[i], c = s_key[l];
                    const unsigned ea = s_ev[i], ec = s_ev[l];
                    if (up ? ev_less(c, ec, a, ea) : ev_less(a, ea, c, ec)) {
                        s_key[i] = c; s_key[l] = a;
                        s_ev[i] = ec; s_ev[l] = ea;
                    }
                }
                __syncthreads();
            }
        }
        for (int k = tid; k < mc; k += nt) A[c0 + k] = s_ev[k];
        __syncthreads();
    }
    // pairwise merges of the runs
    unsigned *src = A, *dst = scratch;
    for (unsigned L = SEG_CAP; L < m; L <<= 1) {
        for (unsigned r0 = 0; r0 < m; r0 += 2 * L) {
            const int la = (int)min(L, m - r0);
            const int lb = (int)min(L, m - r0 - la);
            const unsigned *ra = src + r0, *rb = src + r0 + la;
            unsigned *o = dst + r0;
            const long long T = (long long)la + lb;
            const int d0 = (int)(T * tid / nt), d1 = (int)(T * (tid + 1) / nt);
            auto split = [&](int d) {
                int lo = max(0, d - lb), hi = min(d, la);
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const unsigned x = ra[mid], y = rb[d - 1 - mid];
                    if (ev_less(event_key<G>(xy, x), x, event_key<G>(xy, y), y)) lo = mid + 1;
                    else hi = mid;
                }
                return lo;
            };
            int ia = split(d0), ib = d0 - ia;
            long long ka = ia < la ? event_key<G>(xy, ra[ia]) : KEY_INF;
            long long kb = ib < lb ? event_key<G>(xy, rb[ib]) : KEY_INF;
            for (int d = d0; d < d1; ++d) {
                const bool take_a = ib >= lb || (ia < la && ev_less(ka, ra[ia], kb, rb[ib]));
                if (take_a) {
                    o[d] = ra[ia];
                    ++ia;
                    ka = ia < la ? event_key<G>(xy, ra[ia]) : KEY_INF;
                } else {
                    o[d] = rb[ib];
                    ++ib;
                    kb = ib < lb ? event_key<G>(xy, rb[ib]) : KEY_INF;
                }
            }
        }
        __syncthreads();
        unsigned *t = src; src = dst; dst = t;
    }
    if (src != A) {
        for (unsigned k = tid; k < m; k += nt) A[k] = src[k];
        __syncthreads();
    }
    // group flags; decoding ignores the halves' order, so neighbours may
    // be rewritten concurrently
    for (unsigned k = tid; k < m; k += nt) {
        const unsigned e = A[k];
        const bool c = k > 0 && event_key<G>(xy, A[k - 1]) == event_key<G>(xy, e);
        A[k] = ev_pack(ev_i(e), ev_j(e), c);
    }
    __syncthreads();
}

template <class G>
__global__ void __launch_bounds__(1024) k_segsort_big(const void *__restrict__ xy, unsigned *__restrict__ ev,
                                                      unsigned *__restrict__ ev2,
                                                      const unsigned *__restrict__ base,
                                                      const int *__restrict__ meta,
                                                      const int *__restrict__ oversize)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_spl[SB_MAX];
    __shared__ unsigned s_cnt[SB_MAX + 1], s_cur[SB_MAX];
    __shared__ long long s_kmin[32], s_kmax[32];
    __shared__ int s_F;
    const int nbig = meta[2];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int b = oversize[q];
        const unsigned off = base[b], m = base[b + 1] - off;
        unsigned *A = ev + off, *C = ev2 + off;
        // splitters from a sorted sample of the bucket's keys
        long long *sw = reinterpret_cast<long long *>(smem);
        cta_fill_merge_sort<SB_SAMPLE / 1024>(sw, sw + SB_SAMPLE, SB_SAMPLE, [&](int k) {
            return event_key<G>(xy, A[(unsigned)(((unsigned long long)k * m) / SB_SAMPLE)]);
        });
        if (tid == 0) s_F = (int)min((unsigned)SB_MAX, (m + SB_TARGET - 1) / SB_TARGET);
        __syncthreads();
        const int F = s_F;
        for (int j = tid; j < F - 1; j += nt) s_spl[j] = sw[((j + 1) * SB_SAMPLE) / F];
        for (int j = tid; j <= F; j += nt) s_cnt[j] = 0u;
        __syncthreads();
        auto sub_of = [&](long long key) {   // splitters <= key
            int lo = 0, hi = F - 1;
            while (lo < hi) {
                const int md = (lo + hi) >> 1;
                if (s_spl[md] <= key) lo = md + 1; else hi = md;
            }
            return lo;
        };
        // counts per sub-bucket, least and largest key
        long long kmn = KEY_INF, kmx = -KEY_INF;
        for (unsigned k = tid; k < m; k += nt) {
            const long long key = event_key<G>(xy, A[k]);
            kmn = min(kmn, key);
            kmx = max(kmx, key);
            atomicAdd(&s_cnt[sub_of(key)], 1u);
        }
        for (int s = 16; s >= 1; s >>= 1) {
            kmn = min(kmn, __shfl_xor_sync(FULL, kmn, s));
            kmx = max(kmx, __shfl_xor_sync(FULL, kmx, s));
        }
        if (lane == 0) { s_kmin[warp] = kmn; s_kmax[warp] = kmx; }
        __syncthreads();
        if (tid == 0) {
            unsigned run = 0;
            for (int j = 0; j < F; ++j) {
                const unsigned c = s_cnt[j];
                s_cnt[j] = run;
                s_cur[j] = run;
                run += c;
            }
            s_cnt[F] = run;
            long long a = s_kmin[0], z = s_kmax[0];
            for (int w = 1; w < (int)(nt >> 5); ++w) { a = min(a, s_kmin[w]); z = max(z, s_kmax[w]); }
            s_kmin[0] = a;
            s_kmax[0] = z;
        }
        __syncthreads();
        // the events grouped by sub-bucket into ev2
        for (unsigned k = tid; k < m; k += nt) {
            const unsigned e = A[k];
            C[atomicAdd(&s_cur[sub_of(event_key<G>(xy, e))], 1u)] = e;
        }
        __syncthreads();
        const long long kmin = s_kmin[0], kmax = s_kmax[0];
        for (int j = 0; j < F; ++j) {
            const unsigned a0 = s_cnt[j], a1 = s_cnt[j + 1], mj = a1 - a0;
            if (mj == 0) continue;
            const long long lo = j == 0 ? kmin : s_spl[j - 1];
            // kmax < KEY_INF (events have finite keys), so kmax + 1 does not overflow
            const long long hi = j == F - 1 ? kmax + 1 : s_spl[j];
            bool done = false;
            if (mj <= (unsigned)SEG_CAP)
                done = sort_bucket_words<G>(xy, C + a0, A + a0, mj, lo,
                                            (unsigned long long)hi - (unsigned long long)lo, smem);
            if (!done) {
                // copy back, then the merge fallback in place (scratch: C)
                for (unsigned k = tid; k < mj; k += nt) A[a0 + k] = C[a0 + k];
                __syncthreads();
                sort_big_merge<G>(xy, A + a0, C + a0, mj, smem);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- plan
constexpr unsigned SNAP_SCAN = 4096;   // events searched for a group start before the bucket start is taken

// Last event at or before t that starts a group of equal slopes (t itself if
// it does), found by one warp inside t's bucket: a range then begins with a
// whole group, which its start sort applies at once (a long group of one
// slope costs nothing to sweep there).  A group never spans two buckets, so
// the bucket's first event is always a valid answer; it is taken when no
// start turns up within SNAP_SCAN events.  Every lane returns the same value.
__device__ unsigned snap_group_start(const unsigned *__restrict__ ev, const unsigned *__restrict__ base, int NB,
                                     unsigned t, int lane)
{
    const unsigned E = base[NB];
    if (t >= E) return E;
    int lo = 0, hi = NB;   // base[lo] <= t < base[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= t) lo = mid; else hi = mid;
    }
    const long long bs = base[lo];
    for (long long top = (long long)t + 1; top > bs && (long long)t + 1 - top < SNAP_SCAN; top -= 32) {
        const long long u = top - 32 + lane;
        const unsigned bal = __ballot_sync(FULL, u >= bs && u < top && !ev_cont(ev[u]));
        if (bal) return (unsigned)(top - 32 + (31 - __clz(bal)));
    }
    return (unsigned)bs;
}

// Range r covers the events [s(E r / W), s(E (r + 1) / W)), s = the snap to
// a group start below: equal event counts up to the group granularity.  One
// warp per range.
__global__ void k_plan(const unsigned *__restrict__ ev, const unsigned *__restrict__ base,
                       const int *__restrict__ meta, int W, unsigned *__restrict__ range)
{
    const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (r >= W) return;
    const int NB = meta[0] + 1;
    const unsigned E = base[NB];
    const unsigned a = snap_group_start(ev, base, NB, (unsigned)((unsigned long long)E * r / W), lane);
    const unsigned b = (r == W - 1) ? E
                                    : snap_group_start(ev, base, NB, (unsigned)((unsigned long long)E * (r + 1) / W), lane);
    if (lane == 0) {
        range[2 * r] = a;
        range[2 * r + 1] = b;
    }
}

// Caller-written range bounds (any event offsets) moved to group starts, one
// warp per bound; equal bounds move alike, so adjacent ranges stay adjacent.
__global__ void k_snap_ranges(const unsigned *__restrict__ ev, const unsigned *__restrict__ base,
                              const int *__restrict__ meta, int count, unsigned *__restrict__ range)
{
    const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (k >= count) return;
    const unsigned v = snap_group_start(ev, base, meta[0] + 1, range[k], lane);
    if (lane == 0) range[k] = v;
}

// The snapped bounds are group starts but need not be monotone: a bound
// deep inside a group longer than SNAP_SCAN events moves to its bucket's
// start, one near the group's start to the group's start.  A running maximum over
// the bounds in order (start_0, end_0, start_1, ...) makes them monotone:
// every value is still a group start, a raised start only drops events that
// the previous range already covers, and the ranges become disjoint, so every
// event is swept exactly once (k_sweep checks the total).  One CTA, in
// chunks of consecutive bounds per thread.
__global__ void __launch_bounds__(1024) k_monotone_ranges(unsigned *__restrict__ range, int count)
{
    __shared__ unsigned s_warp[32];
    const int per = (count + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per, k1 = min(count, k0 + per);
    unsigned m = 0;
    for (int k = k0; k < k1; ++k) m = max(m, range[k]);
    // exclusive running maximum of the chunks before this thread's
    unsigned v = m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v = max(v, o);
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(FULL, t, d);
            if (lane >= d) t = max(t, o);
        }
        s_warp[lane] = t;
    }
    __syncthreads();
    unsigned run = __shfl_up_sync(FULL, v, 1);
    if (lane == 0) run = 0u;
    if (warp > 0) run = max(run, s_warp[warp - 1]);
    for (int k = k0; k < k1; ++k) {
        run = max(run, range[k]);
        range[k] = run;
    }
}

// ---------------------------------------------------------------- init
// Bitonic sort of P (power of two) packed words in `a` by one CTA.
__device__ void cta_bitonic_u64(unsigned long long *a, int P)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const unsigned long long x0 = a[i], x1 = a[l];
                if ((x0 > x1) == up) { a[i] = x1; a[l] = x0; }
            }
            __syncthreads();
        }
    }
}

// Bitonic sort of P words in a with a 16-bit payload moved alongside (one
// CTA, global or shared memory).
__device__ void cta_bitonic_kv(unsigned long long *a, unsigned short *pay, int P)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const unsigned long long x0 = a[i], x1 = a[l];
                if ((x0 > x1) == up) {
                    a[i] = x1; a[l] = x0;
                    const unsigned short p0 = pay[i];
                    pay[i] = pay[l]; pay[l] = p0;
                }
            }
            __syncthreads();
        }
    }
}

// Packed sort word of one point at the start slope: (key + 2^32) in bits
// 63..31, (2^15 - 1 - x) in bits 30..15, point index in bits 14..0.
// Ascending words order the points by projection, then x descending, then
// index: the order just after the slope (a line of that slope lists its
// points by decreasing x), which is the order once the range's first group
// of events has been applied.  For int16 points |key| < 2^32 and
// n <= 32768 here, so the fields never overlap.
__device__ __forceinline__ unsigned long long order_word(long long key, int x, int k)
{
    return ((unsigned long long)(key + (1LL << 32)) << 31) | ((unsigned long long)(unsigned)(32767 - x) << 15) |
           (unsigned long long)(unsigned)k;
}

template <bool XY_SMEM>
__device__ unsigned group_end(const int *s_xy, const int *__restrict__ g_xy, const unsigned *__restrict__ ev,
                              unsigned known, unsigned end, int dy0, int dx0, int lane);
__device__ __forceinline__ long long word_key(unsigned long long w) { return (long long)(w >> 31) - (1LL << 32); }
__device__ __forceinline__ int word_index(unsigned long long w) { return (int)(w & 0x7fffu); }

// Start of a sweep range: the points sorted in the order just after the
// range's first slope, every window scored at that slope (with the smallest
// pair of its group), and the range's start moved past that first group:
// its events only reverse the blocks of equal projections, which the
// just-after order already does, and a window's width at the slope does not
// depend on the order inside a block.  The events of the skipped group count
// as covered (meta[7]).
__global__ void __launch_bounds__(1024) k_sweep_init(const int *__restrict__ xy, int n, int h,
                                                     const unsigned *__restrict__ ev,
                                                     unsigned *__restrict__ range, int W,
                                                     int *__restrict__ meta_mut,
                                                     const unsigned *__restrict__ base,
                                                     unsigned short *__restrict__ orders,
                                                     unsigned long long *__restrict__ gsort,
                                                     Cand *__restrict__ cands)
{
    const int *meta = meta_mut;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_w[32];
    __shared__ int s_a[32];
    __shared__ unsigned s_pair[32];
    __shared__ int s_slope[2];
    const int w = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned E = base[meta[0] + 1];
    const unsigned start = range[2 * w], end = range[2 * w + 1];
    const bool vertical = (E == 0 && w == 0);
    if (w == 0 && threadIdx.x == 0) {
        meta_mut[4] = 0;          // range counter of k_sweep
        meta_mut[8] = (int)E;     // events to cover (checked by the final reduction)
    }
    if (start >= end && !vertical) {
        if (threadIdx.x == 0) cands[w] = cand_empty();
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    // global sort space above SORT_SMEM_N points: 2 P words per range (the
    // chunked sort's two buffers), then W P 16-bit payloads
    unsigned long long *a = (n <= SORT_SMEM_N) ? reinterpret_cast<unsigned long long *>(smem)
                                               : gsort + (size_t)w * 2 * P;
    // the slope of the first event (the vertical fallback uses slope 0)
    if (threadIdx.x == 0) {
        int dy = 0, dx = 1;
        if (!vertical) pair_slope(xy[ev_i(ev[start])], xy[ev_j(ev[start])], dy, dx);
        s_slope[0] = dy;
        s_slope[1] = dx;
    }
    __syncthreads();
    const int dy = s_slope[0], dx = s_slope[1];
    // end of the range's first group of equal slopes (warp 0)
    __shared__ unsigned s_g1;
    if (warp == 0) {
        const unsigned g1 = vertical ? end : group_end<false>(nullptr, xy, ev, start + 1, end, dy, dx, lane);
        if (lane == 0) s_g1 = g1;
    }
    auto word = [&](int k) {
        if (k >= n) return ~0ull;
        const int pk = xy[k];
        return order_word(proj(pk, dy, dx), px(pk), k);
    };
    // above 32768 points the index needs 16 bits: the word then holds
    // (key + 2^32, 2^15 - 1 - x) and the index travels in a payload array (equal
    // words are identical points, whose order is immaterial)
    // Above SORT_SMEM_N points, when the projections at the slope span less
    // than 2^32: words (Z - Zmin) << 32 | (32767 - x) << 16 | index, sorted
    // in 8192-word chunks in shared memory and merged in global memory.
    long long zmin = 0;
    bool compact = false;
    if (n > SORT_SMEM_N) {
        long long mn = LLONG_MAX, mx = LLONG_MIN;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const long long z = proj(xy[k], dy, dx);
            mn = min(mn, z);
            mx = max(mx, z);
        }
        for (int m = 16; m >= 1; m >>= 1) {
            mn = min(mn, __shfl_xor_sync(FULL, mn, m));
            mx = max(mx, __shfl_xor_sync(FULL, mx, m));
        }
        __shared__ long long s_mn[32], s_mx[32];
        if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; }
        __syncthreads();
        mn = s_mn[0];
        mx = s_mx[0];
        for (int k = 1; k < nw; ++k) { mn = min(mn, s_mn[k]); mx = max(mx, s_mx[k]); }
        zmin = mn;
        compact = mx - mn < (1LL << 32);
    }
    const bool wide = !compact && n > 32768;
    unsigned short *pay = wide ? reinterpret_cast<unsigned short *>(gsort + (size_t)W * 2 * P) + (size_t)w * P
                               : nullptr;
    if (compact) {
        auto cword = [&](int k) -> unsigned long long {
            if (k >= n) return ~0ull;
            const int pk = xy[k];
            return ((unsigned long long)(proj(pk, dy, dx) - zmin) << 32) |
                   ((unsigned long long)(unsigned)(32767 - px(pk)) << 16) | (unsigned long long)(unsigned)k;
        };
        a = cta_sort_chunked<8192>(reinterpret_cast<unsigned long long *>(smem), a, a + P, P, cword);
    } else if (wide) {
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            if (k < n) {
                const int pk = xy[k];
                a[k] = ((unsigned long long)(proj(pk, dy, dx) + (1LL << 32)) << 16) | (unsigned)(32767 - px(pk));
            } else {
                a[k] = ~0ull;
            }
            pay[k] = (unsigned short)k;
        }
        __syncthreads();
        cta_bitonic_kv(a, pay, P);
    } else if (n > SORT_SMEM_N ||
               !cta_fill_merge_sort_any(a, a + (P < (int)blockDim.x ? (int)blockDim.x : P),
                                        P < (int)blockDim.x ? (int)blockDim.x : P, word)) {
        for (int k = threadIdx.x; k < P; k += blockDim.x) a[k] = word(k);
        __syncthreads();
        cta_bitonic_u64(a, P);
    }
    auto akey = [&](int q) {
        return compact ? (long long)(a[q] >> 32) + zmin
                       : (wide ? (long long)(a[q] >> 16) - (1LL << 32) : word_key(a[q]));
    };
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        orders[(size_t)w * n + k] =
            compact ? (unsigned short)(a[k] & 0xffffu) : (wide ? pay[k] : (unsigned short)word_index(a[k]));
    // every window at the first slope
    long long bw = KEY_INF;
    int ba = 0x7fffffff;
    for (int q = threadIdx.x; q + h - 1 < n; q += blockDim.x) {
        const long long wd = akey(q + h - 1) - akey(q);
        if (wd < bw) { bw = wd; ba = q; }
    }
    // the first event of a group carries its smallest index pair
    unsigned mp = 0xffffffffu;
    if (!vertical) {
        const unsigned e = ev[start];
        mp = ((unsigned)ev_i(e) << 16) | (unsigned)ev_j(e);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        long long ow = __shfl_xor_sync(FULL, bw, m);
        int oa = __shfl_xor_sync(FULL, ba, m);
        if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
        mp = min(mp, __shfl_xor_sync(FULL, mp, m));
    }
    if (lane == 0) { s_w[warp] = bw; s_a[warp] = ba; s_pair[warp] = mp; }
    __syncthreads();
    if (warp == 0) {
        bw = lane < nw ? s_w[lane] : KEY_INF;
        ba = lane < nw ? s_a[lane] : 0x7fffffff;
        mp = lane < nw ? s_pair[lane] : 0xffffffffu;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            long long ow = __shfl_xor_sync(FULL, bw, m);
            int oa = __shfl_xor_sync(FULL, ba, m);
            if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
            mp = min(mp, __shfl_xor_sync(FULL, mp, m));
        }
        if (lane == 0) {
            Cand c;
            c.w = bw;
            c.t = akey(ba) + akey(ba + h - 1);
            c.dy = dy;
            c.dx = dx;
            c.i = vertical ? -1 : (int)(mp >> 16);
            c.j = vertical ? -1 : (int)(mp & 0xffffu);
            cands[w] = c;
            if (!vertical) {
                range[2 * w] = s_g1;
                atomicAdd(reinterpret_cast<unsigned *>(meta_mut + 7), s_g1 - start);
            }
        }
    }
}

// ---------------------------------------------------------------- sweep
template <bool XY_SMEM>
__device__ __forceinline__ int load_xy(const int *s_xy, const int *__restrict__ g_xy, int k)
{
    return XY_SMEM ? s_xy[k] : __ldg(&g_xy[k]);
}

__device__ __forceinline__ size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

constexpr int RUN_LANE_MAX = 24;   // runs up to this length are handled by one lane
#ifndef LMS_SWEEP_XY_SMEM_MAX
#define LMS_SWEEP_XY_SMEM_MAX 16384     // the sweep keeps the packed points in shared memory up to this n
#endif

#ifndef SWEEP_SERIAL_DEFAULT
#define SWEEP_SERIAL_DEFAULT false
#endif
constexpr bool SWEEP_SERIAL = SWEEP_SERIAL_DEFAULT;   // every batch one event at a time
#ifndef SWEEP_SERIAL_BELOW
#define SWEEP_SERIAL_BELOW 6
#endif
#ifndef SWEEP_SERIAL_CHUNKS
#define SWEEP_SERIAL_CHUNKS 2
#endif
// A parallel batch costs about as much as several events applied one at a time:
// after a batch that advanced fewer than SERIAL_BELOW events, the next
// SERIAL_CHUNKS batches are applied one event at a time; every further such
// batch in a row doubles that count (up to SERIAL_CHUNKS_MAX), and a batch that
// advances well resets it, so stretches of chained events try few batches.
constexpr int SERIAL_BELOW = SWEEP_SERIAL_BELOW, SERIAL_CHUNKS = SWEEP_SERIAL_CHUNKS;
constexpr int SERIAL_CHUNKS_MAX = 8 * SWEEP_SERIAL_CHUNKS;

// A whole group of one slope dy/dx in one pass over the positions, for
// groups of about n/2 events or more.  Two points with equal projections at
// the slope and different x are joined by an event of the group, so every
// maximal block of two or more positions with equal projections is one line
// of that slope (plus duplicates of its points, whose order is immaterial);
// the group reverses exactly these blocks.  The warp slides a window of 32
// positions over the order (lane l holds position p0 + l), compares each
// key with its neighbours' by shuffles, and finds the blocks ending inside
// the window.  The lane holding a block's end reverses it and re-scores its
// two windows, all such lanes at once (the blocks are disjoint); blocks
// longer than HEAVY_LANE_MAX positions are then reversed by the whole warp,
// one after another.  The key at a position depends only on which block
// holds it, not on the order inside the block, so the window-end keys read
// while other blocks are being reversed are the same before and after; and a
// block never reaches past its end, so the next window's entries can be
// fetched before this window's blocks are rewritten.
constexpr int HEAVY_LANE_MAX = 32;

template <bool XY_SMEM>
__device__ void heavy_scan(unsigned short *order, unsigned short *pos, const int *s_xy,
                           const int *__restrict__ g_xy, int n, int h, int dy, int dx, unsigned gmin, int lane,
                           Cand &best)
{
    auto XY = [&](int k) { return load_xy<XY_SMEM>(s_xy, g_xy, k); };
    Cand c;
    c.dy = dy; c.dx = dx; c.i = (int)(gmin >> 16); c.j = (int)(gmin & 0xffffu);
    auto rescore = [&](int s0, int e0, long long K) {
        if (s0 + h - 1 < n) {
            const long long kt = proj(XY(order[s0 + h - 1]), dy, dx);
            c.w = kt - K; c.t = K + kt;
            if (cand_better(c, best)) best = c;
        }
        if (e0 - h + 1 >= 0) {
            const long long kb = proj(XY(order[e0 - h + 1]), dy, dx);
            c.w = K - kb; c.t = kb + K;
            if (cand_better(c, best)) best = c;
        }
    };
    int open = -1;                 // start of a block still open at p0 (warp-uniform)
    long long kprev = 0;           // key at p0 - 1 (p0 > 0)
    int idx = lane < n ? order[lane] : 0;
    int nidx = 32 + lane < n ? order[32 + lane] : 0;
    int p32 = 32 < n ? order[32] : 0;
    for (int p0 = 0; p0 < n; p0 += 32) {
        const int p = p0 + lane;
        const long long k = p < n ? proj(XY(idx), dy, dx) : 0;
        const long long k32 = p0 + 32 < n ? proj(XY(p32), dy, dx) : 0;
        // prefetch the next window (its entries are not rewritten below)
        idx = nidx;
        nidx = p0 + 64 + lane < n ? order[p0 + 64 + lane] : 0;
        p32 = p0 + 64 < n ? order[p0 + 64] : 0;
        long long kn = __shfl_down_sync(FULL, k, 1);
        if (lane == 31) kn = k32;
        long long kp = __shfl_up_sync(FULL, k, 1);
        if (lane == 0) kp = kprev;
        const bool eq_next = p + 1 < n && kn == k;
        const bool eq_prev = p > 0 && p < n && kp == k;
        const unsigned starts = __ballot_sync(FULL, eq_next && !eq_prev);
        const unsigned ends = __ballot_sync(FULL, eq_prev && !eq_next);
        // this lane's block: from the last start at or before it (or the
        // block open since an earlier window) to this lane's end
        const bool is_end = (ends >> lane) & 1u;
        int s0 = -1;
        if (is_end) {
            const unsigned before = starts & ((2u << lane) - 1u);
            s0 = before ? p0 + 31 - __clz(before) : open;
        }
        const int e0 = p0 + lane;
        const bool mine = is_end && s0 >= 0 && e0 - s0 + 1 <= HEAVY_LANE_MAX;
        const bool longb = is_end && s0 >= 0 && !mine;
        __syncwarp();
        if (mine) {
            for (int u = s0, v = e0; u < v; ++u, --v) {
                const unsigned short ou = order[u], ov = order[v];
                order[u] = ov;
                order[v] = ou;
                pos[ov] = (unsigned short)u;
                pos[ou] = (unsigned short)v;
            }
            rescore(s0, e0, k);
        }
        __syncwarp();
        for (unsigned lm = __ballot_sync(FULL, longb); lm; lm &= lm - 1) {
            const int el = __ffs(lm) - 1;
            const int ls0 = __shfl_sync(FULL, s0, el), le0 = p0 + el;
            const long long K = __shfl_sync(FULL, k, el);
            const int len = le0 - ls0 + 1;
            for (int t = lane; t < len / 2; t += 32) {
                const unsigned short u = order[ls0 + t], v = order[le0 - t];
                order[ls0 + t] = v;
                order[le0 - t] = u;
            }
            __syncwarp();
            for (int t = lane; t < len; t += 32) pos[order[ls0 + t]] = (unsigned short)(ls0 + t);
            if (lane == 0) rescore(ls0, le0, K);
            __syncwarp();
        }
        // the block left open at the end of this window, if any
        const int last_s = starts ? 31 - __clz(starts) : -1;
        const int last_e = ends ? 31 - __clz(ends) : -1;
        if (last_s > last_e) open = p0 + last_s;
        else if (ends) open = -1;
        kprev = __shfl_sync(FULL, k, 31);
    }
    __syncwarp();
}

// Slope of event e as (dy, dx), dx > 0.
template <bool XY_SMEM>
__device__ __forceinline__ void event_slope(const int *s_xy, const int *__restrict__ g_xy, unsigned e, int &dy,
                                            int &dx)
{
    pair_slope(load_xy<XY_SMEM>(s_xy, g_xy, ev_i(e)), load_xy<XY_SMEM>(s_xy, g_xy, ev_j(e)), dy, dx);
}

// End of the group of equal slopes dy0/dx0 that starts at g0 and holds at
// least the events [g0, known).  Events are in slope order, so "same slope"
// holds on [g0, g1) and fails on [g1, end): a galloping search (lane l
// probes known + 32 (2^l - 1)), then 33-way bisections, all lanes at once.
template <bool XY_SMEM>
__device__ unsigned group_end(const int *s_xy, const int *__restrict__ g_xy, const unsigned *__restrict__ ev,
                              unsigned known, unsigned end, int dy0, int dx0, int lane)
{
    auto same = [&](unsigned q) {
        int dy, dx;
        event_slope<XY_SMEM>(s_xy, g_xy, ev[q], dy, dx);
        return (long long)dy * dx0 == (long long)dy0 * dx;
    };
    // most groups end within the next 32 events: one coalesced look first
    {
        const unsigned q = known + lane;
        const unsigned out = __ballot_sync(FULL, q < end && !ev_cont(ev[q]));
        if (out) return known + __ffs(out) - 1;
        if (known + 32 >= end) return end;
        known += 32;
    }
    // lo: last index known inside the group; hi: first index known outside
    unsigned lo = known - 1, hi = end;
    {
        const unsigned long long off = 32ull * ((1ull << lane) - 1ull);
        const unsigned long long q = (unsigned long long)known + off;
        const bool in = q < hi && same((unsigned)q);
        const unsigned bal = __ballot_sync(FULL, in);
        const unsigned out = __ballot_sync(FULL, q < hi && !in);
        if (bal) lo = (unsigned)(known + 32ull * ((1ull << (31 - __clz(bal))) - 1ull));
        if (out) hi = (unsigned)(known + 32ull * ((1ull << (__ffs(out) - 1)) - 1ull));
    }
    while (hi - lo > 1) {
        const unsigned span = hi - lo;
        const unsigned q = lo + (unsigned)(((unsigned long long)span * (lane + 1)) / 33);
        const bool valid = q > lo && q < hi;
        const bool in = valid && same(q);
        const unsigned bal = __ballot_sync(FULL, in);
        const unsigned out = __ballot_sync(FULL, valid && !in);
        if (bal) lo = __shfl_sync(FULL, q, 31 - __clz(bal));
        if (out) hi = __shfl_sync(FULL, q, __ffs(out) - 1);
        if (!bal && !out) break;   // span < 33 with no probe strictly inside: cannot happen for span > 1
    }
    return hi;
}

// A whole group of equal slopes [g0, g1) in work proportional to its
// length (any n).  In the order just before the slope, the points of each
// line of that slope fill a block of consecutive positions (they project
// alike), x ascending.  Exactly one event of the group joins the block's
// first point a to the first point above it with a larger x; the lane that
// reads that event reverses the block (the order just after the slope) and
// re-scores the window starting at the block and the window ending at it.
// Events are examined 32 at a time (reads only, then a warp barrier), then
// the claiming lanes rewrite their blocks (disjoint) and the warp waits
// again.  An event whose block was reversed earlier sees b below a and is
// skipped.  The window-end keys read during the rewrites do not depend on
// the order inside other blocks: all points of a block project alike.
template <bool XY_SMEM>
__device__ void group_claims(unsigned short *order, unsigned short *pos, const int *s_xy,
                             const int *__restrict__ g_xy, int n, int h, const unsigned *__restrict__ ev,
                             unsigned g0, unsigned g1, int lane, Cand &best)
{
    auto XY = [&](int k) { return load_xy<XY_SMEM>(s_xy, g_xy, k); };
    const unsigned e0 = ev[g0];
    int dy, dx;
    pair_slope(XY(ev_i(e0)), XY(ev_j(e0)), dy, dx);
    Cand c;
    c.dy = dy; c.dx = dx; c.i = ev_i(e0); c.j = ev_j(e0);
    unsigned e_next = (g0 + lane < g1) ? ev[g0 + lane] : 0u;
    for (unsigned c0 = g0; c0 < g1; c0 += 32) {
        const unsigned q = c0 + lane;
        const unsigned e = e_next;
        e_next = (q + 32 < g1) ? ev[q + 32] : 0u;
        bool claim = false;
        int pa = 0, pb = 0;
        long long K = 0;
        if (q < g1) {
            int Pa = XY(ev_i(e)), Pb = XY(ev_j(e));
            int a = ev_i(e), b = ev_j(e);
            if (px(Pa) > px(Pb)) {
                const int t = a; a = b; b = t;
                const int tp = Pa; Pa = Pb; Pb = tp;
            }
            pa = pos[a];
            pb = pos[b];
            if (pa < pb) {
                K = proj(Pa, dy, dx);
                claim = (pa == 0 || proj(XY(order[pa - 1]), dy, dx) != K) &&
                        (pb == pa + 1 || px(XY(order[pb - 1])) == px(Pa));
            }
        }
        __syncwarp();
        if (claim) {
            int hi = pb;
            while (hi + 1 < n && proj(XY(order[hi + 1]), dy, dx) == K) ++hi;
            for (int u = pa, v = hi; u < v; ++u, --v) {
                const unsigned short ou = order[u], ov = order[v];
                order[u] = ov;
                order[v] = ou;
                pos[ov] = (unsigned short)u;
                pos[ou] = (unsigned short)v;
            }
            if (pa + h - 1 < n) {
                const long long kt = proj(XY(order[pa + h - 1]), dy, dx);
                c.w = kt - K; c.t = K + kt;
                if (cand_better(c, best)) best = c;
            }
            if (hi - h + 1 >= 0) {
                const long long kb = proj(XY(order[hi - h + 1]), dy, dx);
                c.w = K - kb; c.t = kb + K;
                if (cand_better(c, best)) best = c;
            }
        }
        __syncwarp();
    }
}

// One event applied exactly, with the order just before its slope in place.
// Every lane of the warp computes the same values and stores the same words,
// so consecutive events need no barrier; only the cooperative reversal of a
// run (three or more collinear points) is fenced by warp barriers.
//   done    b already sits below a: its run was reversed by an earlier
//           event of the same slope; nothing to do
//   simple  a, b adjacent and both outer neighbours project elsewhere: swap
//   run     the block of positions projecting like a (found by ballots
//           around [pa, pb]) is reversed: the order just after the slope
// The window starting at the lower rewritten position and the window
// ending at the upper one are re-scored (Sec. 3.3: an optimal bracelet has a
// point at one of its ends).
template <bool XY_SMEM>
__device__ __forceinline__ void serial_event(unsigned short *order, unsigned short *pos, const int *s_xy,
                                             const int *__restrict__ g_xy, int n, int h, unsigned e, unsigned gmin,
                                             bool single, int lane, Cand &best, int *err)
{
    auto XY = [&](int k) { return load_xy<XY_SMEM>(s_xy, g_xy, k); };
    int a = ev_i(e), b = ev_j(e);
    int Pa = XY(a), Pb = XY(b);
    int pa = pos[a], pb = pos[b];
    if (px(Pa) > px(Pb)) {
        const int t = a; a = b; b = t;
        const int tp = Pa; Pa = Pb; Pb = tp;
        const int tq = pa; pa = pb; pb = tq;
    }
    if (pb < pa) return;
    const int dx = px(Pb) - px(Pa), dy = py(Pb) - py(Pa);
    const long long K = proj(Pa, dy, dx);
    const int top0 = pa + h - 1, bot0 = pb - h + 1;
    const bool rd_t = top0 < n && top0 > pb, rd_b = bot0 >= 0 && bot0 < pa;
    // single: the pair is alone at its slope, so no neighbour is on its line
    const int i_lo = (!single && pa > 0) ? order[pa - 1] : 0;
    const int i_hi = (!single && pb < n - 1) ? order[pb + 1] : 0;
    const int i_t = rd_t ? order[top0] : 0;
    const int i_b = rd_b ? order[bot0] : 0;
    const bool lo_eq = !single && pa > 0 && proj(XY(i_lo), dy, dx) == K;
    const bool hi_eq = !single && pb < n - 1 && proj(XY(i_hi), dy, dx) == K;
    Cand c;
    c.dy = dy; c.dx = dx; c.i = (int)(gmin >> 16); c.j = (int)(gmin & 0xffffu);
    auto offer = [&](long long wd, long long t) {
        if (best.dx != 0 && wd * (long long)best.dx > best.w * (long long)dx) return;
        c.w = wd; c.t = t;
        if (cand_better(c, best)) best = c;
    };
    if (pb == pa + 1 && !lo_eq && !hi_eq) {
        const long long kt = rd_t ? proj(XY(i_t), dy, dx) : K;
        const long long kb = rd_b ? proj(XY(i_b), dy, dx) : K;
        order[pa] = (unsigned short)b;
        order[pb] = (unsigned short)a;
        pos[b] = (unsigned short)pa;
        pos[a] = (unsigned short)pb;
        if (top0 < n) offer(kt - K, K + kt);
        if (bot0 >= 0) offer(K - kb, kb + K);
        return;
    }
    // a run: extend [pa, pb] over every neighbour projecting like a
    int lo = pa, hi = pb;
    if (lo_eq) {
        lo = pa - 1;
        for (;;) {
            const int q = lo - 1 - lane;
            const unsigned bal = __ballot_sync(FULL, q >= 0 && proj(XY(order[q]), dy, dx) == K);
            if (bal == FULL) { lo -= 32; continue; }
            lo -= __ffs(~bal) - 1;
            break;
        }
    }
    if (hi_eq) {
        hi = pb + 1;
        for (;;) {
            const int q = hi + 1 + lane;
            const unsigned bal = __ballot_sync(FULL, q < n && proj(XY(order[q]), dy, dx) == K);
            if (bal == FULL) { hi += 32; continue; }
            hi += __ffs(~bal) - 1;
            break;
        }
    }
    bool broken = false;
    for (int q = pa + 1 + lane; q < pb; q += 32)
        if (proj(XY(order[q]), dy, dx) != K) broken = true;
    if (__any_sync(FULL, broken) && lane == 0) atomicOr(err, 2);
    const int len = hi - lo + 1;
    __syncwarp();
    for (int t = lane; t < len / 2; t += 32) {
        const unsigned short u = order[lo + t], v = order[hi - t];
        order[lo + t] = v;
        order[hi - t] = u;
    }
    __syncwarp();
    for (int t = lane; t < len; t += 32) pos[order[lo + t]] = (unsigned short)(lo + t);
    __syncwarp();
    const int top = lo + h - 1, bot = hi - h + 1;
    if (top < n) {
        const long long kt = top > hi ? proj(XY(order[top]), dy, dx) : K;
        offer(kt - K, K + kt);
    }
    if (bot >= 0) {
        const long long kb = bot < lo ? proj(XY(order[bot]), dy, dx) : K;
        offer(K - kb, kb + K);
    }
}

// One warp per sweeper; each lane takes one of up to 32 consecutive events.
//
// Invariant: between two event slopes the order is sorted by projection, and
// inside every run of equal projections at an event slope the order is x
// ascending (the order just before the slope).  The just-after order of a
// run is x descending, i.e. the run reversed.
//
// Per event (a, b) with x_a < x_b at slope s:
//   done    b already sits below a: its run was reversed by an earlier event
//           of the same group; nothing to do.
//   simple  a, b adjacent and both outer neighbours project elsewhere: the
//           run is the pair; swap it.
//   run     three or more collinear points: the lane finds the run by
//           comparing projections; the lowest lane of each run (same group,
//           same first position) reverses it.  Runs longer than
//           RUN_LANE_MAX are reversed by the whole warp.
// Every active lane owns the positions [lo, hi] it rewrites and re-scores
// the window starting at lo and the window ending at hi.  Lanes of different
// slopes run in parallel unless an earlier lane's [lo, hi] meets a later
// lane's [lo - 1, hi + 1] or one of its window ends lo + h - 1, hi - h + 1;
// the batch is cut before the first such lane.  All reads of a batch happen
// before its writes.
template <bool XY_SMEM, bool SERIAL = SWEEP_SERIAL>
__global__ void __launch_bounds__(256) k_sweep(const int *__restrict__ g_xy, int n, int h,
                                               const unsigned *__restrict__ ev,
                                               const unsigned *__restrict__ range, int W,
                                               const unsigned short *__restrict__ orders,
                                               Cand *__restrict__ cands, int *__restrict__ meta,
                                               unsigned short *__restrict__ gpos)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int *err = meta + 3;
    unsigned *next_range = reinterpret_cast<unsigned *>(meta + 4);
    int *s_xy = reinterpret_cast<int *>(smem);
    const size_t off0 = XY_SMEM ? align16((size_t)n * 4) : 0;
    const size_t half = align16((size_t)n * 2);
    // order (and, when it fits, pos) of this warp in shared memory; for
    // large n the positions live in the warp's own slice of gpos
    const size_t per = gpos ? half : 2 * half;
    unsigned short *order = reinterpret_cast<unsigned short *>(smem + off0 + warp * per);
    unsigned short *pos = gpos ? gpos + (size_t)(blockIdx.x * nwarp + warp) * n
                               : reinterpret_cast<unsigned short *>(smem + off0 + warp * per + half);
    if (XY_SMEM) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_xy[k] = g_xy[k];
        __syncthreads();
    }
    const int g = blockIdx.x * nwarp + warp;   // this sweeping warp
    // the residue test of the conflict check needs h - 1 >= 8 and n <= 3 (h - 1)
    const int H = h - 1;
    const bool fold_ok = H >= 8 && n <= 3 * H;
    auto XY = [&](int k) { return load_xy<XY_SMEM>(s_xy, g_xy, k); };
    Cand best = cand_empty();
    auto offer = [&](long long wd, long long t, int dy, int dx, unsigned pr) {
        // cheap reject on the width alone before the full lexicographic test
        if (best.dx != 0 && wd * (long long)best.dx > best.w * (long long)dx) return;
        Cand c;
        c.w = wd; c.t = t; c.dy = dy; c.dx = dx;
        c.i = (int)(pr >> 16); c.j = (int)(pr & 0xffffu);
        if (cand_better(c, best)) best = c;
    };
    // ranges are taken in slope order from a shared counter until none is left
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(next_range, 1u);
        w = __shfl_sync(FULL, w, 0);
        if (w >= (unsigned)W) break;
        const unsigned start = range[2 * w], end = range[2 * w + 1];
        if (start >= end) continue;
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned *>(meta + 7), end - start);
        __syncwarp();
        load_order(orders + (size_t)w * n, n, order, pos, lane);
        __syncwarp();
        const unsigned lanemask_le = 0xffffffffu >> (31 - lane);
        const unsigned lanemask_lt = lanemask_le >> 1;
        unsigned carried = 0xffffffffu;   // smallest pair of the group open at k
        int serial_left = SERIAL ? 1 << 30 : 0;   // batches still to be applied one event at a time
        int serial_next = SERIAL_CHUNKS;            // serial batches after the next short parallel one
        unsigned k = start;
        unsigned e_cur = (k + lane < end) ? ev[k + lane] : 0u;
        unsigned e_nxt = (k + 32 + lane < end) ? ev[k + 32 + lane] : 0u;
        while (k < end) {
            const unsigned navail = min(32u, end - k);
            const bool valid = (unsigned)lane < navail;
            const unsigned e = e_cur;
            const bool is_start = valid && !ev_cont(e);
            const unsigned smask = __ballot_sync(FULL, is_start);
            // ---- a long group of one slope starting here: process it whole
            if (smask == 1u && navail == 32u && __shfl_sync(FULL, ev_cont(e_nxt) ? 1 : 0, 0)) {
                const unsigned e0 = __shfl_sync(FULL, e, 0);
                int gdy, gdx;
                event_slope<XY_SMEM>(s_xy, g_xy, e0, gdy, gdx);
                const unsigned g1 = group_end<XY_SMEM>(s_xy, g_xy, ev, k + 33, end, gdy, gdx, lane);
                // one pass over the positions pays off for groups of about n/2 events or more
                if (g1 - k >= (unsigned)n / 2)
                    heavy_scan<XY_SMEM>(order, pos, s_xy, g_xy, n, h, gdy, gdx,
                                        ((unsigned)ev_i(e0) << 16) | (unsigned)ev_j(e0), lane, best);
                else
                    group_claims<XY_SMEM>(order, pos, s_xy, g_xy, n, h, ev, k, g1, lane, best);
                carried = 0xffffffffu;
                k = g1;
                e_cur = (k + lane < end) ? ev[k + lane] : 0u;
                e_nxt = (k + 32 + lane < end) ? ev[k + 32 + lane] : 0u;
                continue;
            }
            if (serial_left > 0) {
                // the events in order, one at a time; a group that starts inside
                // the batch and runs past its end is left to the next batch,
                // which processes it whole
                --serial_left;
                int cnt = (int)navail;
                if (smask > 1u && navail == 32u && __shfl_sync(FULL, ev_cont(e_nxt) ? 1 : 0, 0))
                    cnt = 31 - __clz(smask);
                for (int i = 0; i < cnt; ++i) {
                    const unsigned ei = __shfl_sync(FULL, e, i);
                    const unsigned en = i < 31 ? __shfl_sync(FULL, e, i + 1) : __shfl_sync(FULL, e_nxt, 0);
                    if (!ev_cont(ei)) carried = ((unsigned)ev_i(ei) << 16) | (unsigned)ev_j(ei);
                    serial_event<XY_SMEM>(order, pos, s_xy, g_xy, n, h, ei, carried, !ev_cont(ei) && !ev_cont(en),
                                          lane, best, err);
                }
                const int src = (lane + cnt) & 31;
                const unsigned c1 = __shfl_sync(FULL, e_cur, src);
                const unsigned c2 = __shfl_sync(FULL, e_nxt, src);
                const bool from_cur = lane + cnt < 32;
                k += cnt;
                e_cur = from_cur ? c1 : c2;
                const unsigned q = k + 32 + lane;
                e_nxt = from_cur ? c2 : ((q < end) ? ev[q] : 0u);
                continue;
            }
            const unsigned le = smask & lanemask_le;
            const int gfirst = le ? 31 - __clz(le) : -1;
            const unsigned pairv = ((unsigned)ev_i(e) << 16) | (unsigned)ev_j(e);
            unsigned gmin = __shfl_sync(FULL, pairv, gfirst < 0 ? 0 : gfirst);
            if (gfirst < 0) gmin = carried;
            // ---- analysis (reads only)
            int a = ev_i(e), b = ev_j(e);
            int Pa = XY(a), Pb = XY(b);
            int pa = valid ? pos[a] : 0, pb = valid ? pos[b] : 0;
            if (px(Pa) > px(Pb)) {
                const int t = a; a = b; b = t;
                const int tp = Pa; Pa = Pb; Pb = tp;
                const int tq = pa; pa = pb; pb = tq;
            }
            const int dx = px(Pb) - px(Pa), dy = py(Pb) - py(Pa);
            const bool done = valid && pb < pa;
            const bool live = valid && !done;
            const long long K = proj(Pa, dy, dx);
            // outer neighbours and, for a simple swap, the two window ends, all
            // read at once
            const int top0 = pa + h - 1, bot0 = pb - h + 1;
            const bool rd_t = live && top0 < n && top0 > pb, rd_b = live && bot0 >= 0 && bot0 < pa;
            // A pair alone at its slope has no third point on its line (that
            // point would pair with both at the same slope), so its outer
            // neighbours need no test.  The next event of the last lane is the
            // first of the next batch; past the range end (a group start)
            // events read as 0, a start.
            const unsigned e_dn = __shfl_down_sync(FULL, e, 1), e_n0 = __shfl_sync(FULL, e_nxt, 0);
            const bool single = is_start && !ev_cont(lane == 31 ? e_n0 : e_dn);
            const bool nb = live && !single;
            const int i_lo = (nb && pa > 0) ? order[pa - 1] : 0;
            const int i_hi = (nb && pb < n - 1) ? order[pb + 1] : 0;
            const int i_t = rd_t ? order[top0] : 0;
            const int i_b = rd_b ? order[bot0] : 0;
            const bool lo_eq = nb && pa > 0 && proj(XY(i_lo), dy, dx) == K;
            const bool hi_eq = nb && pb < n - 1 && proj(XY(i_hi), dy, dx) == K;
            long long kt = rd_t ? proj(XY(i_t), dy, dx) : K;
            long long kb = rd_b ? proj(XY(i_b), dy, dx) : K;
            int lo = pa, hi = pb;
            bool simple = false, run = false, longrun = false, interior_bad = false;
            if (live) {
                if (pb == pa + 1 && !lo_eq && !hi_eq) {
                    simple = true;
                } else {
                    run = true;
                    if (lo_eq) {
                        --lo;
                        while (lo > 0 && hi - lo < RUN_LANE_MAX && proj(XY(order[lo - 1]), dy, dx) == K) --lo;
                    }
                    if (hi_eq) {
                        ++hi;
                        while (hi < n - 1 && hi - lo < RUN_LANE_MAX && proj(XY(order[hi + 1]), dy, dx) == K) ++hi;
                    }
                    longrun = hi - lo >= RUN_LANE_MAX;
                    // the two points must sit inside one run; if an earlier lane of
                    // this batch is still to move a point in between, the lane waits
                    for (int q = pa + 1; q < pb && !longrun; ++q)
                        if (proj(XY(order[q]), dy, dx) != K) { interior_bad = true; break; }
                    // window ends of the whole run
                    const int top = lo + h - 1, bot = hi - h + 1;
                    kt = (top < n && top > hi) ? proj(XY(order[top]), dy, dx) : K;
                    kb = (bot >= 0 && bot < lo) ? proj(XY(order[bot]), dy, dx) : K;
                }
            }
            // one leader per run: the lowest lane with the same group and run start
            const unsigned runkey = run ? (((unsigned)lo << 12) | ((unsigned)min(hi - lo, 63) << 6) |
                                           (unsigned)(gfirst + 1))
                                        : (0x80000000u | (unsigned)lane);
            const unsigned peers = __match_any_sync(FULL, runkey);
            const bool leader = run && !longrun && lane == __ffs(peers) - 1;
            const bool act = simple || leader;
            // ---- conflicts with earlier active lanes of other groups
            // A later lane must not read a position an earlier lane of another
            // slope rewrites: its outer neighbours [lo - 1, hi + 1] and its window
            // ends lo + h - 1, hi - h + 1.  (Lanes of one slope never disturb each
            // other: they rewrite disjoint runs and the keys they read do not
            // depend on the order inside a run.)
            const unsigned actm = __ballot_sync(FULL, act);
            const unsigned runm = __ballot_sync(FULL, act && !simple);
            const int top = lo + h - 1, bot = hi - h + 1;
            bool conflict = false;
            if (fold_ok) {
                // Pairs of simple swaps [p, p + 1]: with H = h - 1, earlier e
                // and later l conflict only if e - l lies in [-2, 2]
                // (neighbours), [H - 1, H] (l's window top) or [-H, 1 - H]
                // (l's window bottom): in every case e - l = -2..2 modulo H.
                // So the residues f = p mod H of conflicting lanes are within 2
                // of each other, cyclically, and then share a cell of width 4
                // in one of three grids: f / 4, (f + 2) / 4, ((f + 2) mod H) / 4
                // (the last catches pairs across the wrap).  Lanes sharing a
                // cell are treated as conflicting: a superset, so the cut stays
                // safe.
                const bool sim = act && simple;
                int f = pa;
                if (f >= H) f -= H;
                if (f >= H) f -= H;
                int f2 = f + 2;
                const unsigned none = 0x40000000u | (unsigned)lane;
                const unsigned cA = sim ? (unsigned)(f >> 2) : none;
                const unsigned cB = sim ? (unsigned)(f2 >> 2) : none;
                if (f2 >= H) f2 -= H;
                const unsigned cC = sim ? (unsigned)(f2 >> 2) : none;
                const unsigned grp = __match_any_sync(FULL, (unsigned)(gfirst + 1));
                const unsigned nearm = __match_any_sync(FULL, cA) | __match_any_sync(FULL, cB) |
                                       __match_any_sync(FULL, cC);
                conflict = sim && (nearm & actm & ~runm & ~grp & lanemask_lt) != 0u;
                // Pairs with a run leader (a longer rewritten block), checked
                // exactly in both directions, one leader at a time.
                for (unsigned rm = runm; rm; rm &= rm - 1) {
                    const int t = __ffs(rm) - 1;
                    const int tlo = __shfl_sync(FULL, lo, t), thi = __shfl_sync(FULL, hi, t);
                    const int tg = __shfl_sync(FULL, gfirst, t);
                    const int ttop = tlo + h - 1, tbot = thi - h + 1;
                    const bool other = act && gfirst != tg;
                    // a later lane reads what the leader rewrites
                    if (other && lane > t &&
                        ((tlo <= hi + 1 && thi >= lo - 1) || (top >= tlo && top <= thi) || (bot >= tlo && bot <= thi)))
                        conflict = true;
                    // the leader reads what an earlier lane rewrites
                    const bool hit = other && lane < t &&
                                     ((lo <= thi + 1 && hi >= tlo - 1) || (ttop >= lo && ttop <= hi) ||
                                      (tbot >= lo && tbot <= hi));
                    if (__any_sync(FULL, hit) && lane == t) conflict = true;
                }
            } else {
                const unsigned me = act ? (((unsigned)lo << 16) | ((unsigned)(hi - lo) << 6) | (unsigned)(gfirst + 1))
                                        : 0xffffffffu;
                for (int t = 0; t < 31; ++t) {
                    const unsigned o = __shfl_sync(FULL, me, t);
                    if (!act || t >= lane || o == 0xffffffffu || (o & 0x3fu) == (unsigned)(gfirst + 1)) continue;
                    const int olo = (int)(o >> 16), ohi = olo + (int)((o >> 6) & 0x3ffu);
                    if ((olo <= hi + 1 && ohi >= lo - 1) || (top >= olo && top <= ohi) || (bot >= olo && bot <= ohi))
                        conflict = true;
                }
            }
            const unsigned bad = __ballot_sync(FULL, longrun || interior_bad || conflict);
            int cut = bad ? __ffs(bad) - 1 : (int)navail;
            // a group that starts inside the batch and runs past its end is left
            // to the next batch, which processes it whole
            if (smask > 1u && navail == 32u && __shfl_sync(FULL, ev_cont(e_nxt) ? 1 : 0, 0))
                cut = min(cut, 31 - __clz(smask));
            int advance;
            if (cut > 0) {
                // ---- parallel events: window reads, then the rewrites
                const bool go = act && lane < cut;
                __syncwarp();
                if (go) {
                    if (simple) {
                        order[pa] = (unsigned short)b;
                        order[pa + 1] = (unsigned short)a;
                        pos[b] = (unsigned short)pa;
                        pos[a] = (unsigned short)(pa + 1);
                    } else {
                        for (int u = lo, v = hi; u < v; ++u, --v) {
                            const unsigned short ou = order[u], ov = order[v];
                            order[u] = ov;
                            order[v] = ou;
                            pos[ov] = (unsigned short)u;
                            pos[ou] = (unsigned short)v;
                        }
                    }
                    if (top < n) offer(kt - K, K + kt, dy, dx, gmin);
                    if (bot >= 0) offer(K - kb, kb + K, dy, dx, gmin);
                }
                __syncwarp();
                advance = cut;
            } else {
                // ---- lane 0 holds a long run (or one to verify): the warp reverses it
                const int ra = __shfl_sync(FULL, pa, 0), rb = __shfl_sync(FULL, pb, 0);
                const int rdy = __shfl_sync(FULL, dy, 0), rdx = __shfl_sync(FULL, dx, 0);
                const long long RK = __shfl_sync(FULL, K, 0);
                const unsigned rmin = __shfl_sync(FULL, gmin, 0);
                int rlo = min(ra, rb), rhi = max(ra, rb);
                for (;;) {
                    const int q = rlo - 1 - lane;
                    const bool eq = q >= 0 && proj(XY(order[q]), rdy, rdx) == RK;
                    const unsigned bal = __ballot_sync(FULL, eq);
                    if (bal == FULL) { rlo -= 32; continue; }
                    rlo -= __ffs(~bal) - 1;
                    break;
                }
                for (;;) {
                    const int q = rhi + 1 + lane;
                    const bool eq = q < n && proj(XY(order[q]), rdy, rdx) == RK;
                    const unsigned bal = __ballot_sync(FULL, eq);
                    if (bal == FULL) { rhi += 32; continue; }
                    rhi += __ffs(~bal) - 1;
                    break;
                }
                bool broken = false;
                for (int q = rlo + lane; q <= rhi; q += 32)
                    if (proj(XY(order[q]), rdy, rdx) != RK) broken = true;
                if (__any_sync(FULL, broken) && lane == 0) atomicOr(err, 2);
                const int len = rhi - rlo + 1;
                for (int t = lane; t < len / 2; t += 32) {
                    const unsigned short u = order[rlo + t], v = order[rhi - t];
                    order[rlo + t] = v;
                    order[rhi - t] = u;
                }
                __syncwarp();
                for (int t = lane; t < len; t += 32) pos[order[rlo + t]] = (unsigned short)(rlo + t);
                __syncwarp();
                if (lane == 0) {
                    if (rlo + h - 1 < n) {
                        const long long t2 = proj(XY(order[rlo + h - 1]), rdy, rdx);
                        offer(t2 - RK, RK + t2, rdy, rdx, rmin);
                    }
                    if (rhi - h + 1 >= 0) {
                        const long long b2 = proj(XY(order[rhi - h + 1]), rdy, rdx);
                        offer(RK - b2, b2 + RK, rdy, rdx, rmin);
                    }
                }
                __syncwarp();
                advance = 1;
            }
            carried = __shfl_sync(FULL, gmin, advance - 1);
            // chains of events that share points cut batches short; there one
            // event at a time is cheaper than a parallel step
            if (advance < SERIAL_BELOW) {
                serial_left = serial_next;
                serial_next = min(2 * serial_next, SERIAL_CHUNKS_MAX);
            } else {
                serial_next = SERIAL_CHUNKS;
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
    best = warp_best(best);
    if (lane == 0) cands[W + g] = best;
}

}  // namespace

// ---------------------------------------------------------------- host side
static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Shared memory of one sweep CTA: the points (when kept on chip) plus the
// order and position arrays of each of its sweeping warps.
static size_t sweep_smem_bytes(int n, bool xy_smem, bool pos_smem, int spb)
{
    const size_t per = (pos_smem ? 2 : 1) * (((size_t)n * 2 + 15) / 16 * 16);
    const size_t xyb = xy_smem ? ((size_t)n * 4 + 15) / 16 * 16 : 0;
    return xyb + per * spb;
}

void sweep_plan_configure(SweepPlan &p, int n, int h, int sms, int want_w, int want_b, bool concurrent)
{
    p.n = n;
    p.h = h;
    p.emax = (long long)n * (n - 1) / 2;
    p.xy_smem = n <= LMS_SWEEP_XY_SMEM_MAX;
    // sweeping warps per CTA limited by shared memory (order + pos each;
    // order alone when both do not fit, the positions then in global memory)
    const size_t half = ((size_t)n * 2 + 15) / 16 * 16;
    const size_t xyb = p.xy_smem ? ((size_t)n * 4 + 15) / 16 * 16 : 0;
    const size_t cap = 227 * 1024;
    p.pos_smem = xyb + 2 * half <= cap;
    const size_t per = (p.pos_smem ? 2 : 1) * half;
    int spb = (int)((cap - xyb) / per);
    spb = spb < 1 ? 1 : (spb > 8 ? 8 : spb);
    p.spb = spb;
    // resident sweep CTAs per SM (the sweep kernel is persistent)
    const size_t sw_smem = sweep_smem_bytes(n, p.xy_smem, p.pos_smem, spb);
    int per_sm = 0;
    if (p.xy_smem) {
        cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<true>, 32 * spb, sw_smem);
    } else {
        cudaFuncSetAttribute(k_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<false>, 32 * spb, sw_smem);
    }
    cudaGetLastError();
    if (per_sm < 1) per_sm = 1;
    const long long g_full = (long long)sms * per_sm * spb;
    // slope ranges: RANGE_FACTOR per sweeping warp, handed out dynamically.
    // A range's start sort costs n log n, so ranges hold at least n events
    // where that still keeps every sweeping warp busy (and always when other
    // fits share the GPU), and at least MIN_RANGE_EVENTS events in any case.
    long long w = want_w > 0 ? want_w : RANGE_FACTOR * g_full;
    if (want_w <= 0) {
        const long long by_n = p.emax / (n > MIN_RANGE_EVENTS ? (long long)n : MIN_RANGE_EVENTS) + 1;
        const long long by_min = p.emax / MIN_RANGE_EVENTS + 1;
        const long long cap = concurrent ? by_n : std::max(by_n, std::min(g_full, by_min));
        if (w > cap) w = cap;
    }
    if (w < 1) w = 1;
    p.W = (int)w;
    long long blocks = (w + spb - 1) / spb;
    if (blocks > (long long)sms * per_sm) blocks = (long long)sms * per_sm;
    p.G = (int)(blocks * spb);
    // buckets: ~4K events each, at least 8 samples per bucket
    long long B = want_b > 0 ? want_b : p.emax / 4096 + 1;
    if (B > BND_MAX / 2) B = BND_MAX / 2;
    if (B < 1) B = 1;
    long long S = 8 * B;
    int s2 = SORT_CHUNK;
    while (s2 < S && s2 < (1 << 20)) s2 <<= 1;
    p.S = s2;
    if (B > p.S / 8) B = p.S / 8;
    p.B = (int)B;
    p.C = sms;
    // the kept events of a restricted pass above n = 8192 fill buckets of
    // all pairs far beyond SEG_CAP; below, the resplit costs more than it saves
    p.resplit = n > SORT_SMEM_N;
}

size_t sweep_plan_bytes(const SweepPlan &p)
{
    const int n = p.n, W = p.W, C = p.C, S = p.S;
    const long long emax = (long long)n * (n - 1) / 2;
    int P = 1;
    while (P < n) P <<= 1;
    size_t b = 0;
    b += a256((size_t)n * 4);
    b += 2 * a256((size_t)S * 8);
    b += a256((size_t)BND_MAX * 8);
    b += a256(64);
    b += a256((size_t)C * BND_MAX * 4);
    b += a256((size_t)(BND_MAX + 1) * 4);
    b += a256((size_t)BND_MAX * 4);
    b += a256((size_t)(emax > 0 ? emax : 1) * 4);
    b += a256((size_t)(emax > 0 ? emax : 1) * 4);   // merge copy of large buckets, list of a restricted pass
    b += a256((size_t)2 * W * 4);
    b += a256((size_t)W * n * 2);
    b += (n > SORT_SMEM_N) ? a256((size_t)W * P * 18) : 0;   // start sorts: 2 P words + P payloads per range
    b += a256((size_t)(2 * W + 8) * sizeof(Cand));
    b += p.pos_smem ? 0 : a256((size_t)p.G * n * 2);
    b += a256((size_t)BND_MAX * 8) + a256((size_t)(BND_MAX + 1) * 4) + a256(64);   // resplit buckets
    return b;
}

void sweep_plan_carve(SweepPlan &p, void *ws)
{
    unsigned char *q = static_cast<unsigned char *>(ws);
    int P = 1;
    while (P < p.n) P <<= 1;
    auto take = [&](size_t bytes) { void *r = q; q += a256(bytes); return r; };
    p.xy = (int *)take((size_t)p.n * 4);
    p.skeys = (long long *)take((size_t)p.S * 8);
    p.skeys2 = (long long *)take((size_t)p.S * 8);
    p.bnd = (long long *)take((size_t)BND_MAX * 8);
    p.meta = (int *)take(64);
    p.hist = (unsigned *)take((size_t)p.C * BND_MAX * 4);
    p.base = (unsigned *)take((size_t)(BND_MAX + 1) * 4);
    p.oversize = (int *)take((size_t)BND_MAX * 4);
    p.ev = (unsigned *)take((size_t)(p.emax > 0 ? p.emax : 1) * 4);
    p.ev2 = (unsigned *)take((size_t)(p.emax > 0 ? p.emax : 1) * 4);
    p.range = (unsigned *)take((size_t)2 * p.W * 4);
    p.orders = (unsigned short *)take((size_t)p.W * p.n * 2);
    p.gsort = (p.n > SORT_SMEM_N) ? (unsigned long long *)take((size_t)p.W * P * 18) : nullptr;
    p.cands = (Cand *)take((size_t)(2 * p.W + 8) * sizeof(Cand));
    p.gpos = p.pos_smem ? nullptr : (unsigned short *)take((size_t)p.G * p.n * 2);
    p.bnd2 = (long long *)take((size_t)BND_MAX * 8);
    p.base2 = (unsigned *)take((size_t)(BND_MAX + 1) * 4);
    p.meta2 = (int *)take(64);
}

const long long *sorted_sample(const SweepPlan &p)
{
    return p.S > SAMPLE_CH ? p.skeys2 : p.skeys;
}

// Sorts S sampled keys (a power of two, SORT_CHUNK .. 16 SAMPLE_CH) held in
// keys, scratch beside; returns the array that holds the sorted keys.
static long long *sort_sample(long long *keys, long long *scratch, int S, cudaStream_t st)
{
    const int P = std::min(S, SAMPLE_CH);
    const size_t smem = (size_t)2 * P * 8;
    cudaFuncSetAttribute(k_sort_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    { StageTimer _t(STAGE_SAMPLE_SORT, st); k_sort_chunks<<<S / P, 1024, smem, st>>>(keys, S); }
    if (S <= SAMPLE_CH) return keys;
    { StageTimer _t(STAGE_SAMPLE_SORT, st); k_merge_chunks<<<(S + 255) / 256, 256, 0, st>>>(keys, scratch, S); }
    return scratch;
}

template <class G>
static cudaError_t events_sample(const SweepPlan &p, const void *pts, cudaStream_t st)
{
    const int n = p.n;
    { StageTimer _t(STAGE_SAMPLE, st); k_sample<G><<<(p.S + 255) / 256, 256, 0, st>>>(pts, n, p.emax, p.S, p.skeys); }
    const long long *src = sort_sample(p.skeys, p.skeys2, p.S, st);
    {
        const size_t qs = (size_t)BND_MAX / 2 * 8;
        cudaFuncSetAttribute(k_splitters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qs);
        StageTimer _t(STAGE_SPLITTERS, st);
        k_splitters<<<1, 1024, qs, st>>>(src, p.S, p.B, p.bnd, p.meta);
    }
    return cudaGetLastError();
}

template <class G>
static cudaError_t events_count(const SweepPlan &p, const void *pts, cudaStream_t st)
{
    const size_t cnt_smem = (size_t)BND_MAX * 8 + (size_t)BND_MAX * 4;
    {
        cudaFuncSetAttribute(k_bucket_pairs<false, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
        StageTimer _t(STAGE_COUNT_PAIRS, st);
        k_bucket_pairs<false, G><<<p.C, CNT_THREADS, cnt_smem, st>>>(pts, p.n, p.bnd, p.meta, p.hist, nullptr, nullptr,
                                                                    nullptr);
    }
    { StageTimer _t(STAGE_PREFIX, st); k_bucket_prefix<<<(BND_MAX + 255) / 256, 256, 0, st>>>(p.hist, p.C, p.meta, p.base); }
    { StageTimer _t(STAGE_SCAN, st); k_bucket_scan<<<1, 1024, 0, st>>>(p.base, p.meta); }
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_events_prepare(const SweepPlan &p, const void *pts, cudaStream_t st)
{
    cudaError_t e = events_sample<G>(p, pts, st);
    if (e != cudaSuccess) return e;
    return events_count<G>(p, pts, st);
}

cudaError_t launch_sweep_sample(const SweepPlan &p, const short *x, const short *y, cudaStream_t st)
{
    { StageTimer _t(STAGE_PACK, st); k_pack<<<(p.n + 255) / 256, 256, 0, st>>>(x, y, p.n, p.xy); }
    return events_sample<KeyI16>(p, p.xy, st);
}

size_t band_scratch_bytes(int n)
{
    int P = 1;
    while (P < n) P <<= 1;
    size_t b = a256((size_t)PRE_MAX * n * 8) + a256((size_t)PRE_MAX * 8);
    if (P > 8192) b += a256((size_t)PRE_MAX * 2 * P * 8);
    return b;
}

cudaError_t launch_sweep_count(const SweepPlan &p, const unsigned char *keep, const long long *cov, void *scratch,
                               bool distinct_x, cudaStream_t st)
{
    const int n = p.n;
    int P = 1;
    while (P < n) P <<= 1;
    unsigned char *q = static_cast<unsigned char *>(scratch);
    unsigned long long *words = reinterpret_cast<unsigned long long *>(q);
    q += a256((size_t)PRE_MAX * n * 8);
    long long *band = reinterpret_cast<long long *>(q);
    q += a256((size_t)PRE_MAX * 8);
    unsigned long long *gscr = P > 8192 ? reinterpret_cast<unsigned long long *>(q) : nullptr;
    const size_t cnt_smem = (size_t)BND_MAX * 8 + (size_t)BND_MAX * 4;
    if (n <= TILE_COUNT_MAX_N) {
        cudaFuncSetAttribute(k_tile_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
        StageTimer _t(STAGE_COUNT_PAIRS, st);
        k_tile_pairs<<<p.C, BAND_THREADS, cnt_smem, st>>>(p.xy, n, p.bnd, p.hist, keep, cov, p.meta, p.ev2);
    } else {
        const int Ps = P > 8192 ? 8192 : (P < 1024 ? 1024 : P);
        const size_t sort_smem = (size_t)2 * Ps * 8;
        cudaFuncSetAttribute(k_band_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
        { StageTimer _t(STAGE_COUNT_PAIRS, st); k_band_sort<<<PRE_MAX, 1024, sort_smem, st>>>(p.xy, n, cov, words, band, gscr); }
        cudaFuncSetAttribute(k_band_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
        StageTimer _t(STAGE_COUNT_PAIRS, st);
        k_band_pairs<<<p.C, BAND_THREADS, cnt_smem, st>>>(p.xy, n, p.bnd, p.hist, keep, cov, words, band, p.meta, p.ev2);
    }
    if (distinct_x) {
        cudaFuncSetAttribute(k_distinct_x_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 * 4);
        StageTimer _t(STAGE_OTHER, st);
        k_distinct_x_pairs<<<1, 1024, 32768 * 4, st>>>(p.xy, n, p.meta);
    }
    { StageTimer _t(STAGE_PREFIX, st); k_bucket_prefix<<<(BND_MAX + 255) / 256, 256, 0, st>>>(p.hist, p.C, p.meta, p.base); }
    // without a resplit the list scatter's cursors are these bucket starts
    { StageTimer _t(STAGE_SCAN, st); k_bucket_scan<<<1, 1024, 0, st>>>(p.base, p.meta, p.resplit ? nullptr : p.hist); }
    return cudaGetLastError();
}

cudaError_t launch_sample_counts(const SweepPlan &p, unsigned *counts, cudaStream_t st)
{
    StageTimer _t(STAGE_OTHER, st);
    k_sample_counts<<<(BND_MAX + 255) / 256, 256, 0, st>>>(sorted_sample(p), p.S, p.bnd, p.meta, counts);
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_events_finish(const SweepPlan &p, const void *pts, const unsigned char *keep, cudaStream_t st,
                                 bool plan, bool listed)
{
    const int n = p.n;
    const size_t cnt_smem = (size_t)BND_MAX * 8 + (size_t)BND_MAX * 4;
    cudaFuncSetAttribute(k_bucket_pairs<true, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
    // buckets of the bucket sorts: those of the count, or of a resplit
    const long long *sbnd = p.bnd;
    const unsigned *sbase = p.base;
    int *smeta = p.meta;
    if (listed) {
        // the restricted count listed the kept pairs: place only those
        unsigned *cursor = p.hist;
        const size_t bsm = (size_t)BND_MAX * 8 + (size_t)BND_MAX * 4;
        if (p.resplit) {
            const int S2 = std::min(p.S, RESPLIT_S);
            { StageTimer _t(STAGE_SAMPLE, st); k_list_sample<G><<<(S2 + 255) / 256, 256, 0, st>>>(pts, p.ev2, p.meta + 6, S2, p.skeys); }
            const long long *src = sort_sample(p.skeys, p.skeys2, S2, st);
            {
                StageTimer _t(STAGE_SPLITTERS, st);
                const size_t qs = (size_t)BND_MAX / 2 * 8;
                cudaFuncSetAttribute(k_splitters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qs);
                k_splitters<<<1, 1024, qs, st>>>(src, S2, BND_MAX / 2, p.bnd2, p.meta2, p.meta + 6, RESPLIT_PER);
            }
            if (cudaMemsetAsync(p.base2, 0, (size_t)(BND_MAX + 1) * 4, st) != cudaSuccess) return cudaGetLastError();
            cudaFuncSetAttribute(k_list_hist<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
            { StageTimer _t(STAGE_COUNT_PAIRS, st); k_list_hist<G><<<p.C, CNT_THREADS, bsm, st>>>(pts, p.bnd2, p.meta2, p.ev2, p.meta + 6, p.base2); }
            { StageTimer _t(STAGE_SCAN, st); k_bucket_scan<<<1, 1024, 0, st>>>(p.base2, p.meta2, cursor); }
            sbnd = p.bnd2;
            sbase = p.base2;
            smeta = p.meta2;
        }
        // cursor: the bucket starts, written by the scan of the count (or of the resplit)
        cudaFuncSetAttribute(k_scatter_list<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
        StageTimer _t(STAGE_SCATTER, st);
        k_scatter_list<G><<<p.C, CNT_THREADS, bsm, st>>>(pts, sbnd, smeta, p.ev2, cursor, p.ev, p.meta + 6);
    } else {
        StageTimer _t(STAGE_SCATTER, st);
        k_bucket_pairs<true, G><<<p.C, CNT_THREADS, cnt_smem, st>>>(pts, n, p.bnd, p.meta, p.hist, p.base, p.ev, keep);
    }
    const size_t seg_smem = (size_t)SEG_CAP * 12;
    cudaFuncSetAttribute(k_segsort<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_smem);
    { StageTimer _t(STAGE_SEGSORT, st); k_segsort<G><<<p.C, 1024, seg_smem, st>>>(pts, p.ev, sbase, sbnd, smeta, p.oversize); }
    if (p.emax > SEG_CAP) {
        cudaFuncSetAttribute(k_segsort_big<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_smem);
        StageTimer _t(STAGE_SEGSORT_BIG, st);
        k_segsort_big<G><<<p.C, 1024, seg_smem, st>>>(pts, p.ev, p.ev2, sbase, smeta, p.oversize);
    }
    {
        StageTimer _t(STAGE_PLAN, st);
        if (plan) k_plan<<<(p.W + 7) / 8, 256, 0, st>>>(p.ev, p.base, p.meta, p.W, p.range);
        else k_snap_ranges<<<(2 * p.W + 7) / 8, 256, 0, st>>>(p.ev, p.base, p.meta, 2 * p.W, p.range);
    }
    {
        StageTimer _t(STAGE_PLAN, st);
        k_monotone_ranges<<<1, 1024, 0, st>>>(p.range, 2 * p.W);
    }
    return cudaGetLastError();
}

template cudaError_t launch_events_prepare<KeyF32>(const SweepPlan &, const void *, cudaStream_t);
template cudaError_t launch_events_finish<KeyF32>(const SweepPlan &, const void *, const unsigned char *, cudaStream_t,
                                                  bool, bool);

cudaError_t launch_sweep_prepare(const SweepPlan &p, const short *x, const short *y, cudaStream_t st)
{
    { StageTimer _t(STAGE_PACK, st); k_pack<<<(p.n + 255) / 256, 256, 0, st>>>(x, y, p.n, p.xy); }
    return launch_events_prepare<KeyI16>(p, p.xy, st);
}

cudaError_t launch_sweep_finish(const SweepPlan &p, const unsigned char *keep, cudaStream_t st, bool plan,
                                bool listed)
{
    const int n = p.n;
    cudaError_t e = launch_events_finish<KeyI16>(p, p.xy, keep, st, plan, listed);
    if (e != cudaSuccess) return e;
    int P = 1;
    while (P < n) P <<= 1;
    // words + merge scratch (whole sort, or one 8192-word chunk above SORT_SMEM_N)
    const size_t init_smem = (n <= SORT_SMEM_N) ? (size_t)(P < 1024 ? 1024 : P) * 16 : (size_t)8192 * 16;
    cudaFuncSetAttribute(k_sweep_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)init_smem);
    {
        StageTimer _t(STAGE_INIT, st);
        k_sweep_init<<<p.W, 1024, init_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.meta, p.base, p.orders,
                                                  p.gsort, p.cands);
    }
    const size_t sw_smem = sweep_smem_bytes(n, p.xy_smem, p.pos_smem, p.spb);
    const int blocks = p.G / p.spb;
    if (p.xy_smem) {
        cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        StageTimer _t(STAGE_SWEEP, st);
        k_sweep<true><<<blocks, 32 * p.spb, sw_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.orders, p.cands, p.meta, p.gpos);
    } else {
        cudaFuncSetAttribute(k_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        StageTimer _t(STAGE_SWEEP, st);
        k_sweep<false><<<blocks, 32 * p.spb, sw_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.orders, p.cands, p.meta, p.gpos);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepPlan &p, const short *x, const short *y, cudaStream_t st)
{
    cudaError_t e = launch_sweep_prepare(p, x, y, st);
    if (e != cudaSuccess) return e;
    return launch_sweep_finish(p, nullptr, st, true);
}

}  // namespace lms
