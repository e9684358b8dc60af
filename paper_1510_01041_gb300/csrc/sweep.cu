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
//   sort      sample: shared-memory bitonic chunks + rank merges
//   splitters quantiles of the sample -> slope-bucket boundaries (a key
//             that fills whole quantiles gets a bucket of its own)
//   count     every pair -> bucket, per-CTA shared-memory histograms
//   prefix    per-bucket offsets of each CTA; scan -> bucket starts
//   scatter   every pair -> its bucket (4-byte event)
//   segsort   each bucket sorted by exact slope key in shared memory;
//             the event word records "same slope as previous event"
//   plan      contiguous bucket ranges with equal event counts -> sweepers
//   init      per sweeper: sort the points at its first slope, score every
//             window there
//   sweep     per sweeper (one warp): apply the events in slope order,
//             re-score the touched windows, keep the best
#include "common.cuh"
#include "kernels.cuh"

namespace lms {

namespace {

constexpr long long KEY_INF = 0x7fffffffffffffffLL;
constexpr int TILE = 64;          // pair tile edge of the count / scatter passes
constexpr int CNT_THREADS = 512;  // threads of a count / scatter CTA
constexpr int SORT_CHUNK = 1024;  // sample keys sorted per shared-memory chunk

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
__global__ void k_sample(const int *__restrict__ xy, int n, long long npairs, int S, long long *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const unsigned long long r = mix64(0x5851F42D4C957F2Dull + (unsigned long long)k * 0x9E3779B97F4A7C15ull);
    const long long p = (long long)__umul64hi(r, (unsigned long long)npairs);
    int i, j;
    pair_decode(p, i, j);
    int dy, dx;
    out[k] = pair_slope(xy[i], xy[j], dy, dx) ? slope_key(dy, dx) : KEY_INF;
}

// Bitonic sort of one chunk of SORT_CHUNK keys in shared memory.
__global__ void __launch_bounds__(SORT_CHUNK / 2) k_sort_chunks(long long *__restrict__ keys)
{
    __shared__ long long s[SORT_CHUNK];
    long long *g = keys + (size_t)blockIdx.x * SORT_CHUNK;
    for (int k = threadIdx.x; k < SORT_CHUNK; k += blockDim.x) s[k] = g[k];
    __syncthreads();
    for (int k = 2; k <= SORT_CHUNK; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            const int t = threadIdx.x;
            const int i = 2 * t - (t & (j - 1));
            const int l = i + j;
            const bool up = (i & k) == 0;
            const long long a = s[i], b = s[l];
            if ((a > b) == up) { s[i] = b; s[l] = a; }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < SORT_CHUNK; k += blockDim.x) g[k] = s[k];
}

// Stable merge of neighbouring sorted runs of length `width` by ranking.
__global__ void k_merge_runs(const long long *__restrict__ src, long long *__restrict__ dst, int S, int width)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    const int run = k / width, p = k - run * width;
    const int pair_base = (run & ~1) * width;
    const long long v = src[k];
    const long long *other = src + (size_t)(run ^ 1) * width;
    int lo = 0, hi = width;
    if ((run & 1) == 0) {          // left run: count right elements < v
        while (lo < hi) { int m = (lo + hi) >> 1; if (other[m] < v) lo = m + 1; else hi = m; }
    } else {                       // right run: count left elements <= v
        while (lo < hi) { int m = (lo + hi) >> 1; if (other[m] <= v) lo = m + 1; else hi = m; }
    }
    dst[pair_base + p + lo] = v;
}

// ---------------------------------------------------------------- splitters
// Quantiles of the sorted sample become boundaries; a value that spans two
// or more quantile positions is a heavy slope and gets the singleton bucket
// [v, v + 1).  Boundaries are strictly increasing; the array is padded with
// KEY_INF to the power of two P2 > nbnd.
__global__ void __launch_bounds__(1024) k_splitters(const long long *__restrict__ sorted, int S, int B,
                                                    long long *__restrict__ bnd, int *__restrict__ meta)
{
    __shared__ int s_m;
    __shared__ int s_scan[1024];
    if (threadIdx.x == 0) {
        int lo = 0, hi = S;
        while (lo < hi) { int m = (lo + hi) >> 1; if (sorted[m] < KEY_INF) lo = m + 1; else hi = m; }
        s_m = lo;
    }
    __syncthreads();
    const int m = s_m;
    const int nq = (m > 0) ? B - 1 : 0;          // quantiles b = 1 .. B-1
    const int per = (nq + blockDim.x - 1) / blockDim.x;
    const int b0 = 1 + threadIdx.x * per;
    auto q = [&](int b) { return sorted[(long long)b * m / B]; };
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
    if (threadIdx.x == 0) { meta[0] = nbnd; meta[1] = P2; meta[2] = 0; meta[3] = 0; }
}

// ---------------------------------------------------------------- count / scatter
// Both passes walk the same upper-triangle tiles in the same static order,
// so the scatter's per-CTA bucket cursors match the counts exactly.
template <bool SCATTER>
__global__ void __launch_bounds__(CNT_THREADS) k_bucket_pairs(const int *__restrict__ xy, int n,
                                                              const long long *__restrict__ bnd,
                                                              const int *__restrict__ meta,
                                                              unsigned *__restrict__ hist,
                                                              const unsigned *__restrict__ base,
                                                              unsigned *__restrict__ ev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_bnd = reinterpret_cast<long long *>(smem);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(smem + BND_MAX * sizeof(long long));
    __shared__ int s_tile[TILE];
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
        __syncthreads();
        if (threadIdx.x < TILE) {
            const int j = bj * TILE + threadIdx.x;
            s_tile[threadIdx.x] = j < n ? xy[j] : 0;
        }
        __syncthreads();
        const int i = bi * TILE + il;
        if (i >= n) continue;
        const int pi = xy[i];
#pragma unroll 4
        for (int jj = 0; jj < JPT; ++jj) {
            const int j = bj * TILE + jl0 + jj;
            if (j <= i || j >= n) continue;
            int dy, dx;
            if (!pair_slope(pi, s_tile[jl0 + jj], dy, dx)) continue;
            const int b = bucket_of(s_bnd, P2, slope_key(dy, dx));
            const unsigned slot = atomicAdd(&s_cnt[b], 1u);
            if (SCATTER) ev[slot] = ev_pack(i, j, false);
        }
    }
    if (!SCATTER) {
        __syncthreads();
        for (int k = threadIdx.x; k < NB; k += blockDim.x) my_hist[k] = s_cnt[k];
    }
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
__global__ void __launch_bounds__(1024) k_bucket_scan(unsigned *__restrict__ base, const int *__restrict__ meta)
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
        run += v;
    }
    if (threadIdx.x == 1023) base[NB] = s[1023];
}

// ---------------------------------------------------------------- segsort
__device__ __forceinline__ long long event_key(const int *__restrict__ xy, unsigned e)
{
    int dy, dx;
    pair_slope(__ldg(&xy[ev_i(e)]), __ldg(&xy[ev_j(e)]), dy, dx);
    return slope_key(dy, dx);
}

// Sort each bucket by exact slope key; buckets with more than SEG_CAP
// events are listed for k_segsort_big.
__global__ void __launch_bounds__(1024) k_segsort(const int *__restrict__ xy, unsigned *__restrict__ ev,
                                                  const unsigned *__restrict__ base,
                                                  const long long *__restrict__ bnd, int *__restrict__ meta,
                                                  int *__restrict__ oversize)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *s_key = reinterpret_cast<long long *>(smem);
    unsigned *s_ev = reinterpret_cast<unsigned *>(smem + SEG_CAP * sizeof(long long));
    const int NB = meta[0] + 1;
    for (int b = blockIdx.x; b < NB; b += gridDim.x) {
        const unsigned off = base[b], m = base[b + 1] - off;
        if (m == 0) continue;
        const bool singleton = (b > 0 && b < NB - 1 && bnd[b] == bnd[b - 1] + 1);
        if (m == 1 || singleton) {
            for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
                const unsigned e = ev[off + k];
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
        __syncthreads();
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            if (k < (int)m) {
                const unsigned e = ev[off + k];
                s_key[k] = event_key(xy, e);
                s_ev[k] = e;
            } else {
                s_key[k] = KEY_INF;
                s_ev[k] = 0;
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
                    if ((a > c) == up && a != c) {
                        s_key[i] = c; s_key[l] = a;
                        const unsigned te = s_ev[i]; s_ev[i] = s_ev[l]; s_ev[l] = te;
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

// Fallback for buckets above SEG_CAP: an in-place bitonic sort in global
// memory with keys recomputed from the points.  Every merge starts with a
// flip step, so all compare-exchanges are ascending and the virtual +inf
// padding above m never has to move: exchanges that reach past m are skipped.
__global__ void __launch_bounds__(1024) k_segsort_big(const int *__restrict__ xy, unsigned *__restrict__ ev,
                                                      const unsigned *__restrict__ base,
                                                      const int *__restrict__ meta,
                                                      const int *__restrict__ oversize)
{
    const int nbig = meta[2];
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int b = oversize[q];
        const unsigned off = base[b], m = base[b + 1] - off;
        unsigned *a = ev + off;
        unsigned P = 1;
        while (P < m) P <<= 1;
        for (unsigned k = 2; k <= P; k <<= 1) {
            for (unsigned t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const unsigned half = k >> 1, blk = t / half, r = t - blk * half;
                const unsigned i = blk * k + r, l = blk * k + k - 1 - r;
                if (l >= m) continue;
                const unsigned ea = a[i], eb = a[l];
                if (event_key(xy, ea) > event_key(xy, eb)) { a[i] = eb; a[l] = ea; }
            }
            __syncthreads();
            for (unsigned j = k >> 2; j >= 1; j >>= 1) {
                for (unsigned t = threadIdx.x; t < P / 2; t += blockDim.x) {
                    const unsigned i = 2 * t - (t & (j - 1));
                    const unsigned l = i + j;
                    if (l >= m) continue;
                    const unsigned ea = a[i], eb = a[l];
                    if (event_key(xy, ea) > event_key(xy, eb)) { a[i] = eb; a[l] = ea; }
                }
                __syncthreads();
            }
        }
        // group flags; decoding ignores the halves' order, so neighbours may
        // be rewritten concurrently
        for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
            const unsigned e = a[k];
            const bool c = k > 0 && event_key(xy, a[k - 1]) == event_key(xy, e);
            a[k] = ev_pack(ev_i(e), ev_j(e), c);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- plan
// Sweeper w takes the buckets whose first event falls in [E w / W, E (w+1) / W).
__global__ void k_plan(const unsigned *__restrict__ base, const int *__restrict__ meta, int W,
                       unsigned *__restrict__ range)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const int NB = meta[0] + 1;
    const unsigned E = base[NB];
    auto lb = [&](unsigned long long t) {
        int lo = 0, hi = NB;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (base[mid] < t) lo = mid + 1; else hi = mid; }
        return base[lo];
    };
    range[2 * w] = lb((unsigned long long)E * w / W);
    range[2 * w + 1] = (w == W - 1) ? E : lb((unsigned long long)E * (w + 1) / W);
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

// Packed sort word: (key + 2^33) << 16 | point index; ascending words sort by
// key (then index).  |key| <= 2^32 for int16 points.
__device__ __forceinline__ unsigned long long order_word(long long key, int k)
{
    return ((unsigned long long)(key + (1LL << 33)) << 16) | (unsigned)k;
}
__device__ __forceinline__ long long word_key(unsigned long long w) { return (long long)(w >> 16) - (1LL << 33); }

__global__ void __launch_bounds__(1024) k_sweep_init(const int *__restrict__ xy, int n, int h,
                                                     const unsigned *__restrict__ ev,
                                                     const unsigned *__restrict__ range, int W,
                                                     const int *__restrict__ meta,
                                                     const unsigned *__restrict__ base,
                                                     unsigned short *__restrict__ orders,
                                                     unsigned long long *__restrict__ gsort,
                                                     Cand *__restrict__ cands)
{
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
    if (start >= end && !vertical) {
        if (threadIdx.x == 0) cands[w] = cand_empty();
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    unsigned long long *a = (n <= SORT_SMEM_N) ? reinterpret_cast<unsigned long long *>(smem)
                                               : gsort + (size_t)w * P;
    // the slope of the first event (the vertical fallback uses slope 0)
    if (threadIdx.x == 0) {
        int dy = 0, dx = 1;
        if (!vertical) pair_slope(xy[ev_i(ev[start])], xy[ev_j(ev[start])], dy, dx);
        s_slope[0] = dy;
        s_slope[1] = dx;
    }
    __syncthreads();
    const int dy = s_slope[0], dx = s_slope[1];
    for (int k = threadIdx.x; k < P; k += blockDim.x)
        a[k] = k < n ? order_word(proj(xy[k], dy, dx), k) : ~0ull;
    __syncthreads();
    cta_bitonic_u64(a, P);
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        orders[(size_t)w * n + k] = (unsigned short)(a[k] & 0xffffu);
    // every window at the first slope
    long long bw = KEY_INF;
    int ba = 0x7fffffff;
    for (int q = threadIdx.x; q + h - 1 < n; q += blockDim.x) {
        const long long wd = word_key(a[q + h - 1]) - word_key(a[q]);
        if (wd < bw) { bw = wd; ba = q; }
    }
    // smallest index pair of the first group of equal slopes
    unsigned mp = 0xffffffffu;
    if (!vertical && warp == 0) {
        for (unsigned base_k = start;; base_k += 32) {
            const unsigned k = base_k + lane;
            unsigned e = 0;
            bool member = false;
            if (k < end) {
                e = ev[k];
                member = (k == start) || ev_cont(e);
            }
            const unsigned bal = __ballot_sync(FULL, member);
            const int valid = (bal == FULL) ? 32 : __ffs(~bal) - 1;
            if (lane < valid) mp = min(mp, ((unsigned)ev_i(e) << 16) | (unsigned)ev_j(e));
            if (bal != FULL) break;
        }
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
            c.t = word_key(a[ba]) + word_key(a[ba + h - 1]);
            c.dy = dy;
            c.dx = dx;
            c.i = vertical ? -1 : (int)(mp >> 16);
            c.j = vertical ? -1 : (int)(mp & 0xffffu);
            cands[w] = c;
        }
    }
}

// ---------------------------------------------------------------- sweep
struct SweepSmem {
    unsigned short *order, *pos;
    unsigned *bm;
};

template <bool XY_SMEM>
__device__ __forceinline__ int load_xy(const int *s_xy, const int *__restrict__ g_xy, int k)
{
    return XY_SMEM ? s_xy[k] : __ldg(&g_xy[k]);
}

__device__ __forceinline__ size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// One warp per sweeper.  Lane 0 applies simple events (two points meet);
// the whole warp handles groups of equal slopes (collinear points).
template <bool XY_SMEM>
__global__ void __launch_bounds__(256) k_sweep(const int *__restrict__ g_xy, int n, int h,
                                               const unsigned *__restrict__ ev,
                                               const unsigned *__restrict__ range, int W,
                                               const unsigned short *__restrict__ orders,
                                               Cand *__restrict__ cands, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int nwords = (n + 31) >> 5;
    int *s_xy = reinterpret_cast<int *>(smem);
    const size_t off0 = XY_SMEM ? align16((size_t)n * 4) : 0;
    const size_t per = 2 * align16((size_t)n * 2) + align16((size_t)nwords * 4);
    unsigned short *order = reinterpret_cast<unsigned short *>(smem + off0 + warp * per);
    unsigned short *pos = order + align16((size_t)n * 2) / 2;
    unsigned *bm = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(pos) + align16((size_t)n * 2));
    if (XY_SMEM) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) s_xy[k] = g_xy[k];
        __syncthreads();
    }
    const int w = blockIdx.x * nwarp + warp;
    if (w >= W) return;
    const unsigned start = range[2 * w], end = range[2 * w + 1];
    Cand best = cand_empty();
    if (start < end) {
        for (int a = lane; a < n; a += 32) {
            const unsigned short p = orders[(size_t)w * n + a];
            order[a] = p;
            pos[p] = (unsigned short)a;
        }
        for (int k = lane; k < nwords; k += 32) bm[k] = 0u;
        __syncwarp();
        auto XY = [&](int k) { return load_xy<XY_SMEM>(s_xy, g_xy, k); };
        auto offer = [&](long long wd, long long t, int dy, int dx, int i, int j) {
            Cand c;
            c.w = wd; c.t = t; c.dy = dy; c.dx = dx; c.i = i; c.j = j;
            if (cand_better(c, best)) best = c;
        };
        // a group of equal slopes: events [g0, g1)
        auto group = [&](unsigned g0, unsigned g1) {
            const unsigned e0 = ev[g0];
            int dy, dx;
            pair_slope(XY(ev_i(e0)), XY(ev_j(e0)), dy, dx);
            unsigned mp = 0xffffffffu;
            for (unsigned k = g0 + lane; k < g1; k += 32) {
                const unsigned e = ev[k];
                const int i = ev_i(e), j = ev_j(e);
                mp = min(mp, ((unsigned)i << 16) | (unsigned)j);
                const int p = pos[i], q = pos[j];
                atomicOr(&bm[p >> 5], 1u << (p & 31));
                atomicOr(&bm[q >> 5], 1u << (q & 31));
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) mp = min(mp, __shfl_xor_sync(FULL, mp, m));
            __syncwarp();
            const int gi = (int)(mp >> 16), gj = (int)(mp & 0xffffu);
            int covered = -1;
            for (int wb = 0; wb < nwords; wb += 32) {
                const unsigned word = (wb + lane < nwords) ? bm[wb + lane] : 0u;
                unsigned nz = __ballot_sync(FULL, word != 0u);
                while (nz) {
                    const int l = __ffs(nz) - 1;
                    nz &= nz - 1;
                    const unsigned wd = __shfl_sync(FULL, word, l);
                    if (lane == 0) {
                        unsigned bits = wd;
                        while (bits) {
                            const int b = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int p = (wb + l) * 32 + b;
                            if (p <= covered) continue;
                            const long long K = proj(XY(order[p]), dy, dx);
                            int lo = p, hi = p;
                            while (lo > 0 && proj(XY(order[lo - 1]), dy, dx) == K) --lo;
                            while (hi + 1 < n && proj(XY(order[hi + 1]), dy, dx) == K) ++hi;
                            covered = hi;
                            // just-after order inside the run: x descending, then index
                            for (int u = lo + 1; u <= hi; ++u) {
                                const unsigned short v = order[u];
                                const int xv = px(XY(v));
                                int t = u - 1;
                                while (t >= lo) {
                                    const unsigned short o = order[t];
                                    const int xo = px(XY(o));
                                    if (xo > xv || (xo == xv && o < v)) break;
                                    order[t + 1] = o;
                                    --t;
                                }
                                order[t + 1] = v;
                            }
                            for (int u = lo; u <= hi; ++u) pos[order[u]] = (unsigned short)u;
                            if (lo + h - 1 < n) {
                                const long long kb = proj(XY(order[lo]), dy, dx);
                                const long long kt = proj(XY(order[lo + h - 1]), dy, dx);
                                offer(kt - kb, kb + kt, dy, dx, gi, gj);
                            }
                            if (hi - h + 1 >= 0) {
                                const long long kb = proj(XY(order[hi - h + 1]), dy, dx);
                                const long long kt = proj(XY(order[hi]), dy, dx);
                                offer(kt - kb, kb + kt, dy, dx, gi, gj);
                            }
                        }
                        bm[wb + l] = 0u;
                    }
                    __syncwarp();
                }
            }
        };
        unsigned k = start;
        while (k < end) {
            const unsigned idx = k + lane;
            const unsigned e = idx < end ? ev[idx] : 0u;
            const unsigned cmask = __ballot_sync(FULL, idx < end && ev_cont(e));
            const unsigned cnt = min(32u, end - k);
            const bool tail_cont = (k + 32 < end) ? ev_cont(ev[k + 32]) : false;
            unsigned t = 0;
            bool jumped = false;
            while (t < cnt) {
                const bool next_cont = (t + 1 < 32) ? ((cmask >> (t + 1)) & 1u) : tail_cont;
                if (!next_cont) {
                    const unsigned et = __shfl_sync(FULL, e, t);
                    int ok = 1;
                    if (lane == 0) {
                        const int u = ev_i(et), v = ev_j(et);
                        const int pu = pos[u], pv = pos[v];
                        if (pu - pv == 1 || pv - pu == 1) {
                            const int Pu = XY(u), Pv = XY(v);
                            int dy, dx;
                            pair_slope(Pu, Pv, dy, dx);
                            const int lo = min(pu, pv);
                            if (px(Pu) > px(Pv)) {
                                order[lo] = (unsigned short)u; order[lo + 1] = (unsigned short)v;
                                pos[u] = (unsigned short)lo; pos[v] = (unsigned short)(lo + 1);
                            } else {
                                order[lo] = (unsigned short)v; order[lo + 1] = (unsigned short)u;
                                pos[v] = (unsigned short)lo; pos[u] = (unsigned short)(lo + 1);
                            }
                            const long long K = proj(Pu, dy, dx);
                            if (lo + h - 1 < n) {
                                const long long kt = proj(XY(order[lo + h - 1]), dy, dx);
                                offer(kt - K, K + kt, dy, dx, u, v);
                            }
                            if (lo - h + 2 >= 0 && lo + 1 < n) {
                                const long long kb = proj(XY(order[lo - h + 2]), dy, dx);
                                offer(K - kb, kb + K, dy, dx, u, v);
                            }
                        } else {
                            ok = 0;   // two points that meet must be neighbours
                            atomicOr(err, 1);
                        }
                    }
                    ok = __shfl_sync(FULL, ok, 0);
                    if (!ok) group(k + t, k + t + 1);
                    __syncwarp();
                    ++t;
                } else {
                    // group [k + t, g1): find its end
                    unsigned g1 = k + t + 1;
                    for (;;) {
                        const unsigned q = g1 + lane;
                        const bool c = q < end && ev_cont(ev[q]);
                        const unsigned bal = __ballot_sync(FULL, c);
                        if (bal == FULL) { g1 += 32; continue; }
                        g1 += __ffs(~bal) - 1;
                        break;
                    }
                    group(k + t, g1);
                    k = g1;
                    jumped = true;
                    break;
                }
            }
            if (!jumped) k += cnt;
        }
    }
    if (lane == 0) cands[W + w] = best;
}

}  // namespace

// ---------------------------------------------------------------- host side
static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

void sweep_plan_configure(SweepPlan &p, int n, int h, int sms, int want_w, int want_b)
{
    p.n = n;
    p.h = h;
    p.emax = (long long)n * (n - 1) / 2;
    p.xy_smem = n <= 16384;
    // sweepers per CTA limited by shared memory (order + pos + bitmap each)
    const size_t per = 2 * ((size_t)n * 2 + 15) / 16 * 16 + ((size_t)(n + 31) / 32 * 4 + 15) / 16 * 16;
    const size_t xyb = p.xy_smem ? ((size_t)n * 4 + 15) / 16 * 16 : 0;
    const size_t cap = 227 * 1024;
    int spb = (int)((cap - xyb) / per);
    spb = spb < 1 ? 1 : (spb > 8 ? 8 : spb);
    p.spb = spb;
    long long w = want_w > 0 ? want_w : (long long)sms * spb;
    const long long by_events = p.emax / 1024 + 1;      // at least ~1K events per sweeper
    if (want_w <= 0 && w > by_events) w = by_events;
    if (w < 1) w = 1;
    p.W = (int)w;
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
}

size_t sweep_plan_bytes(int n, int W, int C, int S)
{
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
    b += a256((size_t)2 * W * 4);
    b += a256((size_t)W * n * 2);
    b += (n > SORT_SMEM_N) ? a256((size_t)W * P * 8) : 0;
    b += a256((size_t)2 * W * sizeof(Cand));
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
    p.range = (unsigned *)take((size_t)2 * p.W * 4);
    p.orders = (unsigned short *)take((size_t)p.W * p.n * 2);
    p.gsort = (p.n > SORT_SMEM_N) ? (unsigned long long *)take((size_t)p.W * P * 8) : nullptr;
    p.cands = (Cand *)take((size_t)2 * p.W * sizeof(Cand));
}

cudaError_t launch_sweep(const SweepPlan &p, const short *x, const short *y, cudaStream_t st)
{
    const int n = p.n;
    k_pack<<<(n + 255) / 256, 256, 0, st>>>(x, y, n, p.xy);
    k_sample<<<(p.S + 255) / 256, 256, 0, st>>>(p.xy, n, p.emax, p.S, p.skeys);
    k_sort_chunks<<<p.S / SORT_CHUNK, SORT_CHUNK / 2, 0, st>>>(p.skeys);
    long long *src = p.skeys, *dst = p.skeys2;
    for (int width = SORT_CHUNK; width < p.S; width <<= 1) {
        k_merge_runs<<<(p.S + 255) / 256, 256, 0, st>>>(src, dst, p.S, width);
        long long *t = src; src = dst; dst = t;
    }
    k_splitters<<<1, 1024, 0, st>>>(src, p.S, p.B, p.bnd, p.meta);
    const size_t cnt_smem = (size_t)BND_MAX * 8 + (size_t)BND_MAX * 4;
    cudaFuncSetAttribute(k_bucket_pairs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
    cudaFuncSetAttribute(k_bucket_pairs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
    k_bucket_pairs<false><<<p.C, CNT_THREADS, cnt_smem, st>>>(p.xy, n, p.bnd, p.meta, p.hist, nullptr, nullptr);
    k_bucket_prefix<<<(BND_MAX + 255) / 256, 256, 0, st>>>(p.hist, p.C, p.meta, p.base);
    k_bucket_scan<<<1, 1024, 0, st>>>(p.base, p.meta);
    k_bucket_pairs<true><<<p.C, CNT_THREADS, cnt_smem, st>>>(p.xy, n, p.bnd, p.meta, p.hist, p.base, p.ev);
    const size_t seg_smem = (size_t)SEG_CAP * 12;
    cudaFuncSetAttribute(k_segsort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_smem);
    k_segsort<<<p.C, 1024, seg_smem, st>>>(p.xy, p.ev, p.base, p.bnd, p.meta, p.oversize);
    k_segsort_big<<<p.C, 1024, 0, st>>>(p.xy, p.ev, p.base, p.meta, p.oversize);
    k_plan<<<(p.W + 255) / 256, 256, 0, st>>>(p.base, p.meta, p.W, p.range);
    int P = 1;
    while (P < n) P <<= 1;
    const size_t init_smem = (n <= SORT_SMEM_N) ? (size_t)P * 8 : 0;
    cudaFuncSetAttribute(k_sweep_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)init_smem);
    k_sweep_init<<<p.W, 1024, init_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.meta, p.base, p.orders,
                                              p.gsort, p.cands);
    const int nwords = (n + 31) / 32;
    const size_t per = 2 * (((size_t)n * 2 + 15) / 16 * 16) + ((size_t)nwords * 4 + 15) / 16 * 16;
    const size_t xyb = p.xy_smem ? ((size_t)n * 4 + 15) / 16 * 16 : 0;
    const size_t sw_smem = xyb + per * p.spb;
    const int blocks = (p.W + p.spb - 1) / p.spb;
    if (p.xy_smem) {
        cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        k_sweep<true><<<blocks, 32 * p.spb, sw_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.orders, p.cands, p.meta + 3);
    } else {
        cudaFuncSetAttribute(k_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw_smem);
        k_sweep<false><<<blocks, 32 * p.spb, sw_smem, st>>>(p.xy, n, p.h, p.ev, p.range, p.W, p.orders, p.cands, p.meta + 3);
    }
    return cudaGetLastError();
}

}  // namespace lms
