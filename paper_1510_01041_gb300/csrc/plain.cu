// plain.cu -- the plain per-slope LMS kernel (Algorithm 1, Sec. 3.4).
//
// For every pairwise slope s = dy/dx (Algorithm 1: all pairwise
// intersections of the dual lines), project all n points (the intersection
// of every dual line with the vertical through the vertex), sort the
// projections and take the narrowest window of h consecutive values (the
// bracelet, Sec. 3.2).  The paper gives each vertex a thread block and a
// shared-memory bitonic sort (Sec. 3.6); here each vertex is one warp that
// keeps all n keys in registers (E per lane) and sorts them with a bitonic
// network whose cross-lane steps are warp shuffles, so no shared memory and
// no block barrier sit on the per-slope path.  Each warp walks a strided
// list of slopes and keeps its best window; the per-warp winners are reduced
// by the argmin kernel (Algorithm 1's final parallel reduction).
//
// Keys are exact: int32 when the coordinate ranges guarantee |key| < 2^31
// (checked per launch on the device), int64 otherwise.
#include "common.cuh"
#include "kernels.cuh"

namespace lms {

// Compare-exchange so that a <= b.
template <typename K>
__device__ __forceinline__ void cx(K &a, K &b)
{
    K lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Bitonic sort of 32*E keys held E per lane.  The network uses the blocked
// index e = lane*E + r; which point starts in which slot does not matter, so
// callers load slot (lane, r) with point r*32 + lane (coalesced, conflict
// free).  After the call lane l holds ranks [l*E, l*E + E) in ascending
// order.  Every merge starts with a "flip" step (e against e ^ (k-1)) so all
// later half-cleaner steps move the minimum to the lower index.
template <int E, typename K>
__device__ __forceinline__ void warp_bitonic(K (&v)[E], int lane)
{
    constexpr int P = 32 * E;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
        // flip step: e pairs with e ^ (k - 1)
        if (k <= E) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int q = r ^ (k - 1);
                if (q > r) cx(v[r], v[q]);
            }
        } else {
            const int lm = k / E - 1;                 // lane mask of the flip
            const bool lower = (lane & (k / (2 * E))) == 0;
            K tmp[E];
#pragma unroll
            for (int r = 0; r < E; ++r) tmp[r] = __shfl_xor_sync(FULL, v[E - 1 - r], lm);
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = lower ? min(v[r], tmp[r]) : max(v[r], tmp[r]);
        }
        // half-cleaners
#pragma unroll
        for (int j = k / 4; j >= 1; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int q = r ^ j;
                    if (q > r) cx(v[r], v[q]);
                }
            } else {
                const int lm = j / E;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    K o = __shfl_xor_sync(FULL, v[r], lm);
                    v[r] = lower ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

template <typename K> __device__ __forceinline__ K key_max();
template <> __device__ __forceinline__ int key_max<int>() { return 0x7fffffff; }
template <> __device__ __forceinline__ long long key_max<long long>() { return 0x7fffffffffffffffLL; }

// Score one slope: returns the narrowest window (first one on ties) as a Cand.
template <int E, typename K>
__device__ __forceinline__ Cand score_slope(const int *s_xy, K *s_buf, int n, int h, int dy, int dx,
                                            int lane)
{
    K v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int k = r * 32 + lane;
        if (k < n) {
            const int p = s_xy[k];
            v[r] = (K)py(p) * (K)dx - (K)px(p) * (K)dy;
        } else {
            v[r] = key_max<K>();
        }
    }
    warp_bitonic<E, K>(v, lane);
    // blocked layout -> shared buffer, then every window a in [0, n-h]
#pragma unroll
    for (int r = 0; r < E; ++r) s_buf[lane * E + r] = v[r];
    __syncwarp();
    long long bw = 0x7fffffffffffffffLL;
    int ba = 0x7fffffff;
    for (int a = lane; a <= n - h; a += 32) {
        const long long w = (long long)s_buf[a + h - 1] - (long long)s_buf[a];
        if (w < bw) { bw = w; ba = a; }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        long long ow = __shfl_xor_sync(FULL, bw, m);
        int oa = __shfl_xor_sync(FULL, ba, m);
        if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
    }
    Cand c;
    c.w = bw;
    c.t = (long long)s_buf[ba] + (long long)s_buf[ba + h - 1];
    c.dy = dy;
    c.dx = dx;
    c.i = -1;
    c.j = -1;
    __syncwarp();
    return c;
}

template <int E>
__global__ void __launch_bounds__(256) k_plain(const short *__restrict__ x, const short *__restrict__ y,
                                               int n, int h, long long npairs, Cand *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_xy = reinterpret_cast<int *>(smem);
    long long *s_buf = reinterpret_cast<long long *>(smem + ((n * 4 + 15) & ~15));
    __shared__ int s_red[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 4) s_red[threadIdx.x] = (threadIdx.x & 1) ? -0x40000000 : 0x3fffffff;
    __syncthreads();
    int xmin = 0x3fffffff, xmax = -0x40000000, ymin = 0x3fffffff, ymax = -0x40000000;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int xx = x[k], yy = y[k];
        s_xy[k] = pack_xy(xx, yy);
        xmin = min(xmin, xx); xmax = max(xmax, xx);
        ymin = min(ymin, yy); ymax = max(ymax, yy);
    }
    atomicMin(&s_red[0], xmin); atomicMax(&s_red[1], xmax);
    atomicMin(&s_red[2], ymin); atomicMax(&s_red[3], ymax);
    __syncthreads();
    xmin = s_red[0]; xmax = s_red[1]; ymin = s_red[2]; ymax = s_red[3];
    // |key| <= max|y| * dx_max + max|x| * |dy|_max
    const long long bound = (long long)max(-ymin, ymax) * (xmax - xmin) +
                            (long long)max(-xmin, xmax) * (ymax - ymin);
    const bool use32 = bound < 0x7fffffffLL;

    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    Cand best = cand_empty();
    if (xmin == xmax) {
        // every x equal: no pairwise slope; the window at slope 0 is reported
        if (gwarp == 0) {
            if (use32) best = score_slope<E, int>(s_xy, reinterpret_cast<int *>(s_buf) + warp * 32 * E, n, h, 0, 1, lane);
            else best = score_slope<E, long long>(s_xy, s_buf + warp * 32 * E, n, h, 0, 1, lane);
            best.i = -1;   // i = -1 with dx != 0 marks the vertical fallback
            best.j = -1;
        }
    } else {
        for (long long p = gwarp; p < npairs; p += nwarps) {
            int i, j;
            pair_decode(p, i, j);
            int dy, dx;
            if (!pair_slope(s_xy[i], s_xy[j], dy, dx)) continue;
            Cand c = use32 ? score_slope<E, int>(s_xy, reinterpret_cast<int *>(s_buf) + warp * 32 * E, n, h, dy, dx, lane)
                           : score_slope<E, long long>(s_xy, s_buf + warp * 32 * E, n, h, dy, dx, lane);
            c.i = i;
            c.j = j;
            if (cand_better(c, best)) best = c;
        }
    }
    if (lane == 0) out[gwarp] = best;
}

int plain_elems(int n)
{
    int e = 1;
    while (32 * e < n) e <<= 1;
    return e;
}

cudaError_t launch_plain(const short *x, const short *y, int n, int h, Cand *cands, int nwarps_total,
                         cudaStream_t st)
{
    const int E = plain_elems(n);
    const int threads = 256, wpb = threads / 32;
    const int blocks = nwarps_total / wpb;
    const size_t smem = ((size_t)n * 4 + 15) / 16 * 16 + (size_t)wpb * 32 * E * sizeof(long long);
    const long long npairs = (long long)n * (n - 1) / 2;
#define LMS_PLAIN_CASE(EE)                                                                     \
    case EE:                                                                                   \
        cudaFuncSetAttribute(k_plain<EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        { StageTimer _t(STAGE_PLAIN, st);                                                      \
        k_plain<EE><<<blocks, threads, smem, st>>>(x, y, n, h, npairs, cands); }                \
        break;
    switch (E) {
        LMS_PLAIN_CASE(1)
        LMS_PLAIN_CASE(2)
        LMS_PLAIN_CASE(4)
        LMS_PLAIN_CASE(8)
        LMS_PLAIN_CASE(16)
        LMS_PLAIN_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef LMS_PLAIN_CASE
    return cudaGetLastError();
}

}  // namespace lms
