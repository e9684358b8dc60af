// hough.cu -- Hough-transform line detection refined by exact LMS (Sec. 5).
//
// The paper follows the standard Hough transform (polar accumulator, coarse
// grid) with an LMS fit of the points that support each accumulator peak.
// Stages, all on the caller's stream except the final plan of the batched
// LMS (its set sizes are data dependent):
//   compact   edge pixels of every image, in raster order, as image-centre
//             coordinates (x - W/2, y - H/2) packed in 32 bits
//   vote      every edge pixel votes once per theta bin t (theta_t = pi t /
//             n_theta) for rho bin floor(rho + n_rho/2), clamped, with
//             rho = x cos_t + y sin_t evaluated as two products rounded
//             separately and one rounded sum (no fused multiply-add), so a
//             CPU recomputes every vote bit for bit from the same tables; a
//             CTA owns a tile of theta bins in shared memory
//   peaks     per image, bins ordered by (votes desc, t asc, rho asc);
//             greedy: take the first bin not within +-nms_theta / +-nms_rho
//             of a taken one, top_k times.  The first top_k + (top_k - 1) *
//             ((2 nms_theta + 1)(2 nms_rho + 1) - 1) bins of that order
//             always contain the answer, so only those are sorted.
//   gather    per peak, the edge pixels with |rho(x, y) - rho_p| <= band
//             (rho_p = bin centre, same rounded arithmetic); near-vertical
//             peaks (|sin| < |cos|) swap x and y; each set is sorted by pixel
//             index so its point order (and the LMS index pair) is fixed
//   fit       exact LMS of every set (batched, see batched.cu)
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr int CH = 16384;          // pixels per compaction chunk
constexpr int TT = 14;             // theta bins per vote CTA (TT * n_rho ints of shared memory)
constexpr int PEAK_SMEM = 16384;   // peak candidates sorted in shared memory

__device__ __forceinline__ int rho_index(int p, float c, float s, int n_rho)
{
    const float xr = (float)(short)(p & 0xffff), yr = (float)(p >> 16);
    const float rho = __fadd_rn(__fmul_rn(xr, c), __fmul_rn(yr, s));
    int r = (int)floorf(__fadd_rn(rho, (float)(n_rho / 2)));
    return min(max(r, 0), n_rho - 1);
}

__global__ void k_edge_count(const unsigned char *__restrict__ img, long long HW, int nchunk,
                             int *__restrict__ cnt)
{
    const int b = blockIdx.y, c = blockIdx.x;
    const unsigned char *im = img + (size_t)b * HW;
    int local = 0;
    for (long long k = (long long)c * CH + threadIdx.x; k < min(HW, (long long)(c + 1) * CH); k += blockDim.x)
        local += im[k] != 0;
    for (int s = 16; s >= 1; s >>= 1) local += __shfl_xor_sync(FULL, local, s);
    __shared__ int s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum, local);
    __syncthreads();
    if (threadIdx.x == 0) cnt[(size_t)b * nchunk + c] = s_sum;
}

// Per image: exclusive scan of chunk counts; chunk offsets are global (all
// images concatenated) and img_off[b] = first edge of image b.
__global__ void k_edge_scan(const int *__restrict__ cnt, int nchunk, int B, long long *__restrict__ coff,
                            long long *__restrict__ img_off)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    for (int b = 0; b < B; ++b) {
        img_off[b] = run;
        for (int c = 0; c < nchunk; ++c) {
            coff[(size_t)b * nchunk + c] = run;
            run += cnt[(size_t)b * nchunk + c];
        }
    }
    img_off[B] = run;
}

// Raster-order write: one warp walks its chunk 32 pixels at a time.
__global__ void k_edge_write(const unsigned char *__restrict__ img, int H, int W, int nchunk,
                             const long long *__restrict__ coff, int *__restrict__ pts)
{
    const int b = blockIdx.y, c = blockIdx.x;
    if (threadIdx.x >= 32) return;
    const long long HW = (long long)H * W;
    const unsigned char *im = img + (size_t)b * HW;
    long long o = coff[(size_t)b * nchunk + c];
    const int lane = threadIdx.x;
    for (long long k0 = (long long)c * CH; k0 < min(HW, (long long)(c + 1) * CH); k0 += 32) {
        const long long k = k0 + lane;
        const bool e = k < HW && k < (long long)(c + 1) * CH && im[k] != 0;
        const unsigned m = __ballot_sync(FULL, e);
        if (e) {
            const int yy = (int)(k / W), xx = (int)(k - (long long)yy * W);
            pts[o + __popc(m & ((1u << lane) - 1u))] = pack_xy(xx - W / 2, yy - H / 2);
        }
        o += __popc(m);
    }
}

__global__ void __launch_bounds__(1024) k_vote(const int *__restrict__ pts, const long long *__restrict__ img_off,
                                               const float *__restrict__ cs, int n_theta, int n_rho,
                                               int *__restrict__ acc)
{
    extern __shared__ int s_acc[];
    const int b = blockIdx.y;
    const int t0 = blockIdx.x * TT, tn = min(TT, n_theta - t0);
    for (int k = threadIdx.x; k < TT * n_rho; k += blockDim.x) s_acc[k] = 0;
    float c[TT], s[TT];
#pragma unroll
    for (int q = 0; q < TT; ++q) {
        c[q] = q < tn ? cs[2 * (t0 + q)] : 0.f;
        s[q] = q < tn ? cs[2 * (t0 + q) + 1] : 0.f;
    }
    __syncthreads();
    const long long a = img_off[b], e = img_off[b + 1];
    for (long long k = a + threadIdx.x; k < e; k += blockDim.x) {
        const int p = pts[k];
#pragma unroll
        for (int q = 0; q < TT; ++q)
            if (q < tn) atomicAdd(&s_acc[q * n_rho + rho_index(p, c[q], s[q], n_rho)], 1);
    }
    __syncthreads();
    int *dst = acc + ((size_t)b * n_theta + t0) * n_rho;
    for (int k = threadIdx.x; k < tn * n_rho; k += blockDim.x) dst[k] = s_acc[k];
}

// Peaks of one image per CTA.  Candidate keys: (65535 - votes) << 32 | t << 16 | r.
__global__ void __launch_bounds__(1024) k_peaks(const int *__restrict__ acc, int n_theta, int n_rho, int top_k,
                                                int nms_t, int nms_r, int *__restrict__ peaks,
                                                unsigned long long *__restrict__ gcand, int gcap,
                                                int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_cand = reinterpret_cast<unsigned long long *>(smem);
    __shared__ int s_hist[4096];
    __shared__ int s_thr, s_n;
    const int b = blockIdx.x;
    const int *A = acc + (size_t)b * n_theta * n_rho;
    const long long nb = (long long)n_theta * n_rho;
    for (int k = threadIdx.x; k < 4096; k += blockDim.x) s_hist[k] = 0;
    __syncthreads();
    for (long long k = threadIdx.x; k < nb; k += blockDim.x) atomicAdd(&s_hist[min(A[k], 4095)], 1);
    __syncthreads();
    const long long need = (long long)top_k + (long long)(top_k - 1) * ((2 * nms_t + 1) * (2 * nms_r + 1) - 1);
    if (threadIdx.x == 0) {
        long long run = 0;
        int thr = 0;
        for (int v = 4095; v >= 0; --v) {
            run += s_hist[v];
            if (run >= need) { thr = v; break; }
        }
        s_thr = max(thr, 1);
        s_n = 0;
    }
    __syncthreads();
    const int thr = s_thr;
    unsigned long long *cand = gcand + (size_t)b * gcap;
    for (long long k = threadIdx.x; k < nb; k += blockDim.x) {
        const int v = A[k];
        if (v >= thr) {
            const int slot = atomicAdd(&s_n, 1);
            if (slot < gcap) {
                const int t = (int)(k / n_rho), r = (int)(k - (long long)t * n_rho);
                cand[slot] = ((unsigned long long)(65535 - min(v, 65535)) << 32) | ((unsigned long long)t << 16) |
                             (unsigned long long)r;
            }
        }
    }
    __syncthreads();
    int m = s_n;
    if (m > gcap) {
        if (threadIdx.x == 0) atomicOr(err, 1);
        m = gcap;
    }
    int P = 1;
    while (P < m) P <<= 1;
    unsigned long long *a = (P <= PEAK_SMEM) ? s_cand : cand;
    if (a == s_cand)
        for (int k = threadIdx.x; k < P; k += blockDim.x) a[k] = k < m ? cand[k] : ~0ull;
    else
        for (int k = m + threadIdx.x; k < P; k += blockDim.x) a[k] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int tq = threadIdx.x; tq < P / 2; tq += blockDim.x) {
                const int i = 2 * tq - (tq & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const unsigned long long x0 = a[i], x1 = a[l];
                if ((x0 > x1) == up) { a[i] = x1; a[l] = x0; }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        int taken = 0;
        int tt[64], rr[64];
        for (int q = 0; q < m && taken < top_k; ++q) {
            const unsigned long long key = a[q];
            const int t = (int)((key >> 16) & 0xffff), r = (int)(key & 0xffff);
            bool ok = true;
            for (int u = 0; u < taken && ok; ++u)
                if (abs(tt[u] - t) <= nms_t && abs(rr[u] - r) <= nms_r) ok = false;
            if (!ok) continue;
            tt[taken] = t;
            rr[taken] = r;
            int *pk = peaks + ((size_t)b * top_k + taken) * 3;
            pk[0] = t; pk[1] = r; pk[2] = 65535 - (int)(key >> 32);
            ++taken;
        }
        for (int u = taken; u < top_k; ++u) {
            int *pk = peaks + ((size_t)b * top_k + u) * 3;
            pk[0] = -1; pk[1] = -1; pk[2] = 0;
        }
    }
}

__device__ __forceinline__ bool in_band(int p, float c, float s, float rho_p, float band)
{
    const float xr = (float)(short)(p & 0xffff), yr = (float)(p >> 16);
    const float rho = __fadd_rn(__fmul_rn(xr, c), __fmul_rn(yr, s));
    return fabsf(__fadd_rn(rho, -rho_p)) <= band;
}

// pass 0: count per (image, peak); pass 1: write with per-set cursors.
template <bool WRITE>
__global__ void k_gather(const int *__restrict__ pts, const long long *__restrict__ img_off,
                         const float *__restrict__ cs, int n_rho, const int *__restrict__ peaks, int top_k,
                         float band, int *__restrict__ cnt, const long long *__restrict__ set_off,
                         int *__restrict__ out_key)
{
    const int b = blockIdx.y;
    __shared__ float s_c[64], s_s[64], s_r[64];
    __shared__ int s_cnt[64];
    for (int q = threadIdx.x; q < top_k; q += blockDim.x) {
        const int *pk = peaks + ((size_t)b * top_k + q) * 3;
        const int t = pk[0];
        s_c[q] = t >= 0 ? cs[2 * t] : 0.f;
        s_s[q] = t >= 0 ? cs[2 * t + 1] : 0.f;
        s_r[q] = t >= 0 ? __fadd_rn((float)(pk[1] - n_rho / 2), 0.5f) : 1e30f;
        s_cnt[q] = 0;
    }
    __syncthreads();
    const long long a = img_off[b], e = img_off[b + 1];
    for (long long k = a + (long long)blockIdx.x * blockDim.x + threadIdx.x; k < e;
         k += (long long)gridDim.x * blockDim.x) {
        const int p = pts[k];
        for (int q = 0; q < top_k; ++q) {
            if (!in_band(p, s_c[q], s_s[q], s_r[q], band)) continue;
            if (WRITE) {
                const int slot = atomicAdd(&cnt[(size_t)b * top_k + q], 1);
                out_key[set_off[(size_t)b * top_k + q] + slot] = (int)(k - a);   // raster rank within the image
            } else {
                atomicAdd(&s_cnt[q], 1);
            }
        }
    }
    if (!WRITE) {
        __syncthreads();
        for (int q = threadIdx.x; q < top_k; q += blockDim.x)
            if (s_cnt[q]) atomicAdd(&cnt[(size_t)b * top_k + q], s_cnt[q]);
    }
}

// Sort every set by raster rank, then emit its coordinates (transposed for
// near-vertical peaks).
__global__ void __launch_bounds__(1024) k_set_finish(const int *__restrict__ pts, const long long *__restrict__ img_off,
                                                     const float *__restrict__ cs, const int *__restrict__ peaks,
                                                     int top_k, const long long *__restrict__ set_off,
                                                     int *__restrict__ keys, short *__restrict__ sx,
                                                     short *__restrict__ sy, int *__restrict__ err)
{
    extern __shared__ int s_k[];
    const int set = blockIdx.x;
    const int b = set / top_k;
    const long long a = set_off[set], m = set_off[set + 1] - a;
    if (m == 0) return;
    int P = 1;
    while (P < m) P <<= 1;
    if (P > 32768) {
        if (threadIdx.x == 0) atomicOr(err, 2);
        return;
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) s_k[k] = k < m ? keys[a + k] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int tq = threadIdx.x; tq < P / 2; tq += blockDim.x) {
                const int i = 2 * tq - (tq & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const int x0 = s_k[i], x1 = s_k[l];
                if ((x0 > x1) == up) { s_k[i] = x1; s_k[l] = x0; }
            }
            __syncthreads();
        }
    }
    const int t = peaks[(size_t)set * 3];
    const float c = cs[2 * t], s = cs[2 * t + 1];
    const bool transpose = fabsf(s) < fabsf(c);
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int p = pts[img_off[b] + s_k[k]];
        const short xx = (short)(p & 0xffff), yy = (short)(p >> 16);
        sx[a + k] = transpose ? yy : xx;
        sy[a + k] = transpose ? xx : yy;
    }
}

// Copy the fitted sets (src offset, count) into consecutive positions.
__global__ void k_compact_sets(const short *__restrict__ sx, const short *__restrict__ sy,
                               const long long *__restrict__ src, const long long *__restrict__ dst,
                               short *__restrict__ tx, short *__restrict__ ty)
{
    const int u = blockIdx.x;
    const long long a = src[u], o = dst[u], m = dst[u + 1] - dst[u];
    for (long long k = threadIdx.x; k < m; k += blockDim.x) {
        tx[o + k] = sx[a + k];
        ty[o + k] = sy[a + k];
    }
}

// SplitMix64's output function (Steele, Lea and Flood, 2014) on a counter:
// the upper 32 bits decide whether point u of set k is kept.
__device__ __forceinline__ unsigned keep_hash(unsigned long long seed, unsigned long long k, unsigned long long u)
{
    unsigned long long z = seed ^ (((k << 32) | u) * 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (unsigned)(z >> 32);
}

// Random subsampling of the fitted sets, one CTA per set: COUNT = true
// writes the kept count of each set, COUNT = false writes the kept points at
// dst (raster order kept: a block-wide rank by ballots).  thr[u] = 0 keeps
// every point.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_subsample(const short *__restrict__ sx, const short *__restrict__ sy,
                                                   const long long *__restrict__ src,
                                                   const long long *__restrict__ cnt,
                                                   const unsigned *__restrict__ thr,
                                                   const int *__restrict__ set_id, unsigned long long seed,
                                                   const long long *__restrict__ dst, int *__restrict__ kept,
                                                   short *__restrict__ tx, short *__restrict__ ty)
{
    __shared__ int s_warp[8];
    const int u = blockIdx.x;
    const long long a = src[u], m = cnt[u];
    const unsigned th = thr[u];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long run = 0;
    for (long long c0 = 0; c0 < m; c0 += blockDim.x) {
        const long long q = c0 + threadIdx.x;
        const bool keep = q < m && (th == 0u || keep_hash(seed, (unsigned long long)set_id[u], (unsigned long long)q) < th);
        const unsigned bal = __ballot_sync(FULL, keep);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += s_warp[w];
            total += s_warp[w];
        }
        if (!COUNT && keep) {
            const long long o = dst[u] + run + before + __popc(bal & ((1u << lane) - 1u));
            tx[o] = sx[a + q];
            ty[o] = sy[a + q];
        }
        run += total;
        __syncthreads();
    }
    if (COUNT && threadIdx.x == 0) kept[u] = (int)run;
}

// Exact sums n, sum x, sum y, sum x^2, sum x y of each fitted set (int16
// points, at most 32768 of them: every sum fits in int64).
__global__ void __launch_bounds__(256) k_ols_sums(const short *__restrict__ tx, const short *__restrict__ ty,
                                                  const long long *__restrict__ dst, long long *__restrict__ sums)
{
    __shared__ long long s_part[8][5];
    const int u = blockIdx.x;
    const long long a = dst[u], m = dst[u + 1] - a;
    long long v[5] = {0, 0, 0, 0, 0};
    for (long long q = threadIdx.x; q < m; q += blockDim.x) {
        const long long x = tx[a + q], y = ty[a + q];
        v[0] += 1; v[1] += x; v[2] += y; v[3] += x * x; v[4] += x * y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
        if (lane == 0) s_part[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w][threadIdx.x];
        sums[5 * (size_t)u + threadIdx.x] = t;
    }
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lms

using namespace lms;

static_assert(sizeof(lms_line) == 136, "lms_line layout");

extern "C" {

// Host tables: theta_t = pi t / n_theta, cos and sin in double rounded to float.
static void make_tables(int n_theta, std::vector<float> &cs)
{
    cs.resize(2 * (size_t)n_theta);
    for (int t = 0; t < n_theta; ++t) {
        const double th = M_PI * (double)t / (double)n_theta;
        cs[2 * t] = (float)cos(th);
        cs[2 * t + 1] = (float)sin(th);
    }
}

int lms_hough_refine(const uint8_t *edges, int64_t B, int32_t H, int32_t W, int32_t n_theta, int32_t n_rho,
                     int32_t top_k, float band_px, int32_t nms_theta, int32_t nms_rho, int32_t max_points,
                     uint64_t sample_seed, const float *cos_sin, int32_t *acc_out, lms_line *out,
                     lms_stream_t stream)
{
    if (!edges || !out || B < 1 || H < 2 || W < 2 || H > 32768 || W > 32768) return LMS_ERR_ARG;
    if (n_theta < 1 || n_theta > 65535 || n_rho < 2 || n_rho > 65535 || top_k < 1 || top_k > 64) return LMS_ERR_ARG;
    if (nms_theta < 0 || nms_rho < 0 || !(band_px >= 0.f) || max_points < 0) return LMS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long HW = (long long)H * W;
    const int nchunk = (int)((HW + CH - 1) / CH);
    const int gcap = 1 << 17;
    // one scratch allocation for everything except the LMS plan
    size_t bytes = 0;
    bytes += a256(sizeof(int) * B * nchunk);                 // chunk counts
    bytes += a256(sizeof(long long) * B * nchunk);           // chunk offsets
    bytes += a256(sizeof(long long) * (B + 1));              // image offsets
    bytes += a256(sizeof(int) * B * HW / 8 + 1024);           // edge points (up to 1/8 of all pixels)
    bytes += acc_out ? 0 : a256(sizeof(int) * B * (size_t)n_theta * n_rho);
    bytes += a256(sizeof(float) * 2 * n_theta);
    bytes += a256(sizeof(int) * 3 * B * top_k);               // peaks
    bytes += a256(sizeof(unsigned long long) * B * gcap);     // peak candidates
    bytes += a256(sizeof(int) * B * top_k);                   // set counts
    bytes += a256(sizeof(long long) * (B * top_k + 1));       // set offsets
    bytes += a256(sizeof(int) * 16);                          // error flags
    unsigned char *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) { cudaGetLastError(); return LMS_ERR_CUDA; }
    unsigned char *q = mem;
    auto take = [&](size_t b) { void *r = q; q += a256(b); return r; };
    int *ccnt = (int *)take(sizeof(int) * B * nchunk);
    long long *coff = (long long *)take(sizeof(long long) * B * nchunk);
    long long *img_off = (long long *)take(sizeof(long long) * (B + 1));
    const long long pts_cap = B * HW / 8 + 256;
    int *pts = (int *)take(sizeof(int) * B * HW / 8 + 1024);
    int *acc = acc_out ? acc_out : (int *)take(sizeof(int) * B * (size_t)n_theta * n_rho);
    float *cs = (float *)take(sizeof(float) * 2 * n_theta);
    int *peaks = (int *)take(sizeof(int) * 3 * B * top_k);
    unsigned long long *gcand = (unsigned long long *)take(sizeof(unsigned long long) * B * gcap);
    int *scnt = (int *)take(sizeof(int) * B * top_k);
    long long *soff = (long long *)take(sizeof(long long) * (B * top_k + 1));
    int *err = (int *)take(sizeof(int) * 16);
    int rc = LMS_OK;
    std::vector<float> hcs;
    if (cos_sin) {
        cudaMemcpyAsync(cs, cos_sin, sizeof(float) * 2 * n_theta, cudaMemcpyDeviceToDevice, st);
    } else {
        make_tables(n_theta, hcs);
        cudaMemcpyAsync(cs, hcs.data(), sizeof(float) * 2 * n_theta, cudaMemcpyHostToDevice, st);
    }
    cudaMemsetAsync(err, 0, sizeof(int) * 16, st);
    cudaMemsetAsync(scnt, 0, sizeof(int) * B * top_k, st);
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_edge_count<<<dim3(nchunk, (unsigned)B), 256, 0, st>>>(edges, HW, nchunk, ccnt);
    }
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_edge_scan<<<1, 32, 0, st>>>(ccnt, nchunk, (int)B, coff, img_off);
    }
    std::vector<long long> hoff(B + 1);
    cudaMemcpyAsync(hoff.data(), img_off, sizeof(long long) * (B + 1), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaFree(mem); return LMS_ERR_CUDA; }
    if (hoff[B] > pts_cap) { cudaFree(mem); return LMS_ERR_UNSUPPORTED; }
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_edge_write<<<dim3(nchunk, (unsigned)B), 32, 0, st>>>(edges, H, W, nchunk, coff, pts);
    }
    const size_t vsm = sizeof(int) * TT * (size_t)n_rho;
    if (vsm > 227 * 1024) { cudaFree(mem); return LMS_ERR_UNSUPPORTED; }
    cudaFuncSetAttribute(k_vote, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm);
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_vote<<<dim3((n_theta + TT - 1) / TT, (unsigned)B), 1024, vsm, st>>>(pts, img_off, cs, n_theta, n_rho, acc);
    }
    cudaFuncSetAttribute(k_peaks, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_SMEM * 8);
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_peaks<<<(unsigned)B, 1024, PEAK_SMEM * 8, st>>>(acc, n_theta, n_rho, top_k, nms_theta, nms_rho, peaks, gcand,
                                                         gcap, err);
    }
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_gather<false><<<dim3(64, (unsigned)B), 256, 0, st>>>(pts, img_off, cs, n_rho, peaks, top_k, band_px, scnt,
                                                              nullptr, nullptr);
    }
    std::vector<int> hcnt(B * top_k), hpk(3 * B * top_k);
    cudaMemcpyAsync(hcnt.data(), scnt, sizeof(int) * B * top_k, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hpk.data(), peaks, sizeof(int) * 3 * B * top_k, cudaMemcpyDeviceToHost, st);
    int herr[2] = {0, 0};
    cudaMemcpyAsync(herr, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaFree(mem); return LMS_ERR_CUDA; }
    if (herr[0]) { cudaFree(mem); return LMS_ERR_UNSUPPORTED; }
    std::vector<long long> hsoff(B * top_k + 1, 0);
    for (long long k = 0; k < B * top_k; ++k) hsoff[k + 1] = hsoff[k] + hcnt[k];
    const long long total = hsoff[B * top_k];
    int *keys = nullptr;
    short *sx = nullptr, *sy = nullptr;
    if (cudaMalloc(&keys, sizeof(int) * std::max(1LL, total)) != cudaSuccess ||
        cudaMalloc(&sx, sizeof(short) * std::max(1LL, total)) != cudaSuccess ||
        cudaMalloc(&sy, sizeof(short) * std::max(1LL, total)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(keys); cudaFree(sx); cudaFree(sy); cudaFree(mem);
        return LMS_ERR_CUDA;
    }
    cudaMemcpyAsync(soff, hsoff.data(), sizeof(long long) * (B * top_k + 1), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(scnt, 0, sizeof(int) * B * top_k, st);
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_gather<true><<<dim3(64, (unsigned)B), 256, 0, st>>>(pts, img_off, cs, n_rho, peaks, top_k, band_px, scnt,
                                                             soff, keys);
    }
    cudaFuncSetAttribute(k_set_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768 * 4);
    {
        StageTimer _t(STAGE_HOUGH, st);
        k_set_finish<<<(unsigned)(B * top_k), 1024, 32768 * 4, st>>>(pts, img_off, cs, peaks, top_k, soff, keys, sx,
                                                                    sy, err);
    }
    // exact LMS of every set of a real peak with at least two points (after
    // the optional subsampling), and the least-squares sums of the same points
    std::vector<int> fit_set;
    std::vector<long long> src, cntv;
    std::vector<unsigned> thr;
    for (long long k = 0; k < B * top_k; ++k) {
        if (hpk[3 * k] < 0 || hcnt[k] < 2) continue;
        fit_set.push_back((int)k);
        src.push_back(hsoff[k]);
        cntv.push_back(hcnt[k]);
        const bool sub = max_points > 0 && hcnt[k] > max_points;
        unsigned t = 0;
        if (sub) {
            t = (unsigned)(((unsigned long long)max_points << 32) / (unsigned long long)hcnt[k]);
            if (t == 0) t = 1;
        }
        thr.push_back(t);
    }
    std::vector<lms_result> res(fit_set.size());
    std::vector<long long> sums(5 * fit_set.size(), 0);
    std::vector<long long> dst(fit_set.size() + 1, 0);
    if (!fit_set.empty()) {
        const size_t F = fit_set.size();
        lms_batch_plan *plan = nullptr;
        long long *d_src = nullptr, *d_dst = nullptr, *d_cnt = nullptr, *d_sums = nullptr;
        unsigned *d_thr = nullptr;
        int *d_id = nullptr, *d_kept = nullptr;
        lms_result *d_res = nullptr;
        short *tx = nullptr, *ty = nullptr;
        const long long all = std::accumulate(cntv.begin(), cntv.end(), 0LL);
        if (cudaMalloc(&d_src, sizeof(long long) * F) != cudaSuccess ||
            cudaMalloc(&d_cnt, sizeof(long long) * F) != cudaSuccess ||
            cudaMalloc(&d_dst, sizeof(long long) * (F + 1)) != cudaSuccess ||
            cudaMalloc(&d_thr, sizeof(unsigned) * F) != cudaSuccess ||
            cudaMalloc(&d_id, sizeof(int) * F) != cudaSuccess ||
            cudaMalloc(&d_kept, sizeof(int) * F) != cudaSuccess ||
            cudaMalloc(&d_sums, sizeof(long long) * 5 * F) != cudaSuccess ||
            cudaMalloc(&d_res, sizeof(lms_result) * F) != cudaSuccess ||
            cudaMalloc(&tx, sizeof(short) * std::max(1LL, all)) != cudaSuccess ||
            cudaMalloc(&ty, sizeof(short) * std::max(1LL, all)) != cudaSuccess) {
            cudaGetLastError();
            rc = LMS_ERR_CUDA;
        }
        if (rc == LMS_OK) {
            cudaMemcpyAsync(d_src, src.data(), sizeof(long long) * F, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(d_cnt, cntv.data(), sizeof(long long) * F, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(d_thr, thr.data(), sizeof(unsigned) * F, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(d_id, fit_set.data(), sizeof(int) * F, cudaMemcpyHostToDevice, st);
            std::vector<int> kept(F);
            if (max_points > 0) {
                {
                    StageTimer _t(STAGE_HOUGH, st);
                    k_subsample<true><<<(unsigned)F, 256, 0, st>>>(sx, sy, d_src, d_cnt, d_thr, d_id, sample_seed,
                                                                   nullptr, d_kept, nullptr, nullptr);
                }
                cudaMemcpyAsync(kept.data(), d_kept, sizeof(int) * F, cudaMemcpyDeviceToHost, st);
                if (cudaStreamSynchronize(st) != cudaSuccess) rc = LMS_ERR_CUDA;
                // a sample of fewer than two points cannot be fitted: keep that set whole
                bool redo = false;
                for (size_t u = 0; u < F; ++u)
                    if (kept[u] < 2) { thr[u] = 0; kept[u] = (int)cntv[u]; redo = true; }
                if (redo) cudaMemcpyAsync(d_thr, thr.data(), sizeof(unsigned) * F, cudaMemcpyHostToDevice, st);
            } else {
                for (size_t u = 0; u < F; ++u) kept[u] = (int)cntv[u];
            }
            for (size_t u = 0; u < F; ++u) dst[u + 1] = dst[u] + kept[u];
        }
        if (rc == LMS_OK) {
            cudaMemcpyAsync(d_dst, dst.data(), sizeof(long long) * (F + 1), cudaMemcpyHostToDevice, st);
            StageTimer _t(STAGE_HOUGH, st);
            k_subsample<false><<<(unsigned)F, 256, 0, st>>>(sx, sy, d_src, d_cnt, d_thr, d_id, sample_seed, d_dst,
                                                            nullptr, tx, ty);
        }
        if (rc == LMS_OK) {
            StageTimer _t(STAGE_HOUGH, st);
            k_ols_sums<<<(unsigned)F, 256, 0, st>>>(tx, ty, d_dst, d_sums);
        }
        if (rc == LMS_OK) rc = lms_batch_plan_create((const int64_t *)dst.data(), (int64_t)F, nullptr, 0, 16, &plan);
        if (rc == LMS_OK) rc = lms_fit_batched(plan, tx, ty, (const int64_t *)d_dst, d_res, stream);
        if (rc == LMS_OK) {
            cudaMemcpyAsync(res.data(), d_res, sizeof(lms_result) * F, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(sums.data(), d_sums, sizeof(long long) * 5 * F, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = LMS_ERR_CUDA;
        }
        lms_batch_plan_destroy(plan);
        cudaFree(d_src); cudaFree(d_dst); cudaFree(d_cnt); cudaFree(d_thr); cudaFree(d_id); cudaFree(d_kept);
        cudaFree(d_sums); cudaFree(d_res); cudaFree(tx); cudaFree(ty);
    }
    std::vector<float> tab(2 * (size_t)n_theta);
    cudaMemcpyAsync(tab.data(), cs, sizeof(float) * 2 * n_theta, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(herr, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == LMS_OK) rc = LMS_ERR_CUDA;
    if (rc == LMS_OK && herr[1]) rc = LMS_ERR_UNSUPPORTED;
    size_t u = 0;
    for (long long k = 0; k < B * top_k; ++k) {
        lms_line &L = out[k];
        memset(&L, 0, sizeof(L));
        L.theta_index = hpk[3 * k];
        L.rho_index = hpk[3 * k + 1];
        L.votes = hpk[3 * k + 2];
        L.npoints = hcnt[k];
        if (L.theta_index >= 0)
            L.transposed = fabsf(tab[2 * L.theta_index + 1]) < fabsf(tab[2 * L.theta_index]) ? 1 : 0;
        L.ols_theta1 = L.ols_theta2 = NAN;
        if (u < fit_set.size() && fit_set[u] == (int)k) {
            L.fit = res[u];
            L.nfit = (int)(dst[u + 1] - dst[u]);
            const long long *S = &sums[5 * u];
            // least squares: theta1 = (n Sxy - Sx Sy) / (n Sxx - Sx^2), exact
            // integers, one double division; theta2 = (Sy - theta1 Sx) / n
            const long long num = S[0] * S[4] - S[1] * S[2], den = S[0] * S[3] - S[1] * S[1];
            if (den != 0 && S[0] > 0) {
                L.ols_theta1 = (double)num / (double)den;
                L.ols_theta2 = ((double)S[2] - L.ols_theta1 * (double)S[1]) / (double)S[0];
            }
            ++u;
        } else {
            L.fit.status = LMS_ERR_ARG;
            L.fit.i = L.fit.j = -1;
        }
    }
    cudaFree(keys); cudaFree(sx); cudaFree(sy); cudaFree(mem);
    return rc;
}

}  // extern "C"
