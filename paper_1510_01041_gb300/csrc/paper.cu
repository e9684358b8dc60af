// paper.cu -- the paper's own three-kernel layout of Algorithm 1 (Sec. 3.4,
// Sec. 3.6), kept as an ablation beside the per-slope warp kernel (plain.cu)
// and the kinetic sweep (sweep.cu).  Same exact integer arithmetic and the
// same tie order as the other paths, so it returns the same bit-exact result.
//
//   K1 vertices   thread blocks of 8 x 8 threads over an (n/8) x (n/8) grid;
//                 thread (i, j) with i > j forms the intersection of dual
//                 lines i and j (the slope of the primal pair); the first row
//                 and column of each block stage the block's 8 + 8 lines in
//                 shared memory; adjacent threads write adjacent records.
//   K2 bracelets  one thread block per vertex, P/2 threads (P = n rounded up
//                 to a power of two, the padding sorts last; at least one
//                 warp); each thread projects two points onto the vertical
//                 through the vertex, the block sorts the P keys with a
//                 shared-memory bitonic network and scans every window of h
//                 consecutive keys.
//   K3 reduction  the exact lexicographic argmin over all vertices
//                 (argmin.cu).
//
// Work is n(n-1)/2 sorts of n keys, O(n^3 log n) as the paper states (Sec.
// 3.5); it is meant for the sizes of the paper's Table 1 (n <= 1024).
#include "common.cuh"
#include "kernels.cuh"

namespace lms {

namespace {

// One vertex of the dual arrangement: slope dy/dx (dx > 0) of the pair
// (i, j), i < j; dx == 0 marks a pair with equal x (no vertex).
struct Vertex {
    int dy, dx, i, j;
};

__global__ void __launch_bounds__(64) k_vertices(const short *__restrict__ x, const short *__restrict__ y, int n,
                                                 Vertex *__restrict__ vert)
{
    __shared__ int s_row[8], s_col[8];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * 8 + ty, j = blockIdx.x * 8 + tx;
    if (tx == 0 && i < n) s_row[ty] = pack_xy(x[i], y[i]);
    if (ty == 0 && j < n) s_col[tx] = pack_xy(x[j], y[j]);
    __syncthreads();
    if (i >= n || j >= n || i <= j) return;
    Vertex v;
    v.i = j;
    v.j = i;
    if (!pair_slope(s_col[tx], s_row[ty], v.dy, v.dx)) v.dx = 0;
    vert[(size_t)i * (i - 1) / 2 + j] = v;
}

// Block k < nv scores vertex k; block nv scores slope 0 when every x is
// equal (no vertex exists) and is empty otherwise.
__global__ void k_bracelets(const short *__restrict__ x, const short *__restrict__ y, int n, int h, int P,
                            const Vertex *__restrict__ vert, long long nv, Cand *__restrict__ out)
{
    extern __shared__ __align__(16) long long s_key[];
    __shared__ long long s_w[32];
    __shared__ int s_a[32];
    __shared__ int s_flat;
    const long long k = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (blockDim.x + 31) >> 5;
    Vertex v;
    if (k < nv) {
        v = vert[k];
    } else {
        // the fallback block: all x equal?
        if (t == 0) s_flat = 1;
        __syncthreads();
        for (int q = t; q < n; q += blockDim.x)
            if (x[q] != x[0]) s_flat = 0;
        __syncthreads();
        v.dy = 0;
        v.dx = s_flat ? 1 : 0;
        v.i = -1;
        v.j = -1;
    }
    if (v.dx == 0) {
        if (t == 0) out[k] = cand_empty();
        return;
    }
    // two projections per thread onto the vertical through the vertex
    for (int q = t; q < P; q += blockDim.x)
        s_key[q] = q < n ? (long long)y[q] * v.dx - (long long)x[q] * v.dy : 0x7fffffffffffffffLL;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int jj = kk >> 1; jj >= 1; jj >>= 1) {
            for (int q = t; q < P / 2; q += blockDim.x) {
                const int a = 2 * q - (q & (jj - 1)), b = a + jj;
                const bool up = (a & kk) == 0;
                const long long ka = s_key[a], kb = s_key[b];
                if ((ka > kb) == up) { s_key[a] = kb; s_key[b] = ka; }
            }
            __syncthreads();
        }
    }
    long long bw = 0x7fffffffffffffffLL;
    int ba = 0x7fffffff;
    for (int a = t; a + h - 1 < n; a += blockDim.x) {
        const long long w = s_key[a + h - 1] - s_key[a];
        if (w < bw) { bw = w; ba = a; }
    }
    for (int m = 16; m >= 1; m >>= 1) {
        const long long ow = __shfl_xor_sync(FULL, bw, m);
        const int oa = __shfl_xor_sync(FULL, ba, m);
        if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
    }
    if (lane == 0) { s_w[warp] = bw; s_a[warp] = ba; }
    __syncthreads();
    if (warp == 0) {
        bw = lane < nw ? s_w[lane] : 0x7fffffffffffffffLL;
        ba = lane < nw ? s_a[lane] : 0x7fffffff;
        for (int m = 16; m >= 1; m >>= 1) {
            const long long ow = __shfl_xor_sync(FULL, bw, m);
            const int oa = __shfl_xor_sync(FULL, ba, m);
            if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
        }
        if (lane == 0) {
            Cand c;
            c.w = bw;
            c.t = s_key[ba] + s_key[ba + h - 1];
            c.dy = v.dy;
            c.dx = v.dx;
            c.i = v.i;
            c.j = v.j;
            out[k] = c;
        }
    }
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t paper_bytes(int n)
{
    const long long nv = (long long)n * (n - 1) / 2;
    return a256((size_t)nv * sizeof(Vertex)) + a256((size_t)(nv + 1) * sizeof(Cand));
}

cudaError_t launch_paper(const short *x, const short *y, int n, int h, void *ws, Cand **cands, long long *count,
                         cudaStream_t st)
{
    const long long nv = (long long)n * (n - 1) / 2;
    Vertex *vert = static_cast<Vertex *>(ws);
    Cand *out = reinterpret_cast<Cand *>(static_cast<unsigned char *>(ws) + a256((size_t)nv * sizeof(Vertex)));
    int P = 2;
    while (P < n) P <<= 1;
    const int g = (n + 7) / 8;
    {
        StageTimer _t(STAGE_PLAIN, st);
        k_vertices<<<dim3(g, g), dim3(8, 8), 0, st>>>(x, y, n, vert);
    }
    {
        StageTimer _t(STAGE_PLAIN, st);
        // whole warps (the reductions shuffle over full warps)
        const int threads = P / 2 < 32 ? 32 : P / 2;
        k_bracelets<<<(unsigned)(nv + 1), threads, (size_t)P * 8, st>>>(x, y, n, h, P, vert, nv, out);
    }
    *cands = out;
    *count = nv + 1;
    return cudaGetLastError();
}

}  // namespace lms
