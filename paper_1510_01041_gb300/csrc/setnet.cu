// setnet.cu -- learned slope proposal: a small set network with BF16 weights
// and FP32 accumulation, its forward, backward and Adam kernels.
//
// The network sees one point set at a time: every point (normalised by the
// set's bounding box) goes through 2 -> 64 -> 64 (ReLU) units, a max over
// the points pools the set into 64 features, and a 64 -> 32 (ReLU) -> 2 head
// predicts the slope angle phi and the intercept b of the LMS line in the
// normalised frame.  Normalisation: cx, cy = bounding-box centres, scale =
// half the larger box side (the same for x and y, so slopes are unchanged).
// The prediction seeds the branch-and-bound's upper bound; the exact search
// never depends on it for correctness.
//
// Parameters (FP32 master copy, BF16 copy used by the forward pass):
//   W1[64][2] b1[64] W2[64][64] b2[64] W3[32][64] b3[32] W4[2][32] b4[2]
// Activations and accumulations are FP32.  The max-pool keeps, per channel,
// the largest value and (on ties) the smallest point index, so the backward
// pass only revisits at most 64 points per set.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr int H1 = 64, H2 = 64, H3 = 32, NOUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H1 * 2, OFF_W2 = OFF_B1 + H1, OFF_B2 = OFF_W2 + H2 * H1,
              OFF_W3 = OFF_B2 + H2, OFF_B3 = OFF_W3 + H3 * H2, OFF_W4 = OFF_B3 + H3,
              OFF_B4 = OFF_W4 + NOUT * H3, NPARAM = OFF_B4 + NOUT;
constexpr int STATE = 8;   // per set: cx, cy, scale, phi, b, slope, theta2, loss

__device__ __forceinline__ float ld(const __nv_bfloat16 *w, int k) { return __bfloat162float(w[k]); }

// per-set normalisation from the bounding box
__device__ void set_frame(const short *x, const short *y, long long a, long long b, float &cx, float &cy,
                          float &sc)
{
    __shared__ int s_b[4];
    if (threadIdx.x < 4) s_b[threadIdx.x] = (threadIdx.x & 1) ? -0x7fffffff : 0x7fffffff;
    __syncthreads();
    int x0 = 0x7fffffff, x1 = -0x7fffffff, y0 = 0x7fffffff, y1 = -0x7fffffff;
    for (long long k = a + threadIdx.x; k < b; k += blockDim.x) {
        x0 = min(x0, (int)x[k]); x1 = max(x1, (int)x[k]);
        y0 = min(y0, (int)y[k]); y1 = max(y1, (int)y[k]);
    }
    atomicMin(&s_b[0], x0); atomicMax(&s_b[1], x1);
    atomicMin(&s_b[2], y0); atomicMax(&s_b[3], y1);
    __syncthreads();
    cx = 0.5f * ((float)s_b[0] + (float)s_b[1]);
    cy = 0.5f * ((float)s_b[2] + (float)s_b[3]);
    sc = 0.5f * fmaxf((float)(s_b[1] - s_b[0]), (float)(s_b[3] - s_b[2]));
    if (sc < 1.0f) sc = 1.0f;
    __syncthreads();
}

// Forward in three launches so that one large set spreads over many SMs.
// Stage 1, one CTA per set: the set's frame into state[0..2]; clears its pool.
__global__ void __launch_bounds__(256) k_setnet_frame(const short *__restrict__ x, const short *__restrict__ y,
                                                      const long long *__restrict__ off, float *__restrict__ state,
                                                      unsigned long long *__restrict__ pool)
{
    const int set = blockIdx.x;
    float cx, cy, sc;
    set_frame(x, y, off[set], off[set + 1], cx, cy, sc);
    if (threadIdx.x == 0) {
        float *st = state + (size_t)set * STATE;
        st[0] = cx; st[1] = cy; st[2] = sc;
    }
    if (threadIdx.x < H2) pool[(size_t)set * H2 + threadIdx.x] = 0ull;
}

// Stage 2, grid (set, slice): the per-point layers over one slice of a set's
// points (slices of whole warps) and the max-pool of the slice, merged into
// the set's pool by atomic maxima.  A pool entry keeps the largest value
// and, on ties, the smallest point index; the maximum does not depend on how
// the points are sliced, so the result is the same for any grid.
__global__ void __launch_bounds__(256) k_setnet_points(const __nv_bfloat16 *__restrict__ wb,
                                                       const short *__restrict__ x, const short *__restrict__ y,
                                                       const long long *__restrict__ off,
                                                       const float *__restrict__ state,
                                                       unsigned long long *__restrict__ pool)
{
    __shared__ float s_w1[H1 * 2], s_b1[H1], s_w2[H2 * H1], s_b2[H2];
    __shared__ unsigned long long s_pool[H2];
    const int set = blockIdx.x;
    const long long a = off[set], b = off[set + 1];
    const long long chunk = ((b - a + gridDim.y - 1) / gridDim.y + 31) & ~31LL;
    const long long c0 = a + chunk * blockIdx.y, c1 = min(b, c0 + chunk);
    if (c0 >= c1) return;
    for (int k = threadIdx.x; k < H1 * 2; k += blockDim.x) s_w1[k] = ld(wb, OFF_W1 + k);
    for (int k = threadIdx.x; k < H1; k += blockDim.x) s_b1[k] = ld(wb, OFF_B1 + k);
    for (int k = threadIdx.x; k < H2 * H1; k += blockDim.x) s_w2[k] = ld(wb, OFF_W2 + k);
    for (int k = threadIdx.x; k < H2; k += blockDim.x) { s_b2[k] = ld(wb, OFF_B2 + k); s_pool[k] = 0ull; }
    const float *st = state + (size_t)set * STATE;
    const float cx = st[0], cy = st[1], sc = st[2];
    const float inv = 1.0f / sc;
    const int lane = threadIdx.x & 31;
    __syncthreads();
    // points: one per lane, warps stride over the slice
    for (long long base = c0 + (threadIdx.x & ~31); base < c1; base += blockDim.x) {
        const long long p = base + lane;
        const bool valid = p < c1;
        const float xn = valid ? ((float)x[p] - cx) * inv : 0.f;
        const float yn = valid ? ((float)y[p] - cy) * inv : 0.f;
        float h1[H1];
#pragma unroll
        for (int k = 0; k < H1; ++k) {
            float acc = s_b1[k];
            acc = fmaf(s_w1[2 * k], xn, acc);
            acc = fmaf(s_w1[2 * k + 1], yn, acc);
            h1[k] = fmaxf(acc, 0.f);
        }
        for (int c = 0; c < H2; ++c) {
            float acc = s_b2[c];
#pragma unroll
            for (int k = 0; k < H1; ++k) acc = fmaf(s_w2[c * H1 + k], h1[k], acc);
            const float h2 = fmaxf(acc, 0.f);
            unsigned long long key = valid ? (((unsigned long long)__float_as_uint(h2) << 32) |
                                              (unsigned long long)(0xffffffffu - (unsigned)(p - a)))
                                           : 0ull;
#pragma unroll
            for (int s2 = 16; s2 >= 1; s2 >>= 1) {
                const unsigned long long o = __shfl_xor_sync(FULL, key, s2);
                key = o > key ? o : key;
            }
            if (lane == 0) atomicMax(&s_pool[c], key);
        }
    }
    __syncthreads();
    if (threadIdx.x < H2) atomicMax(&pool[(size_t)set * H2 + threadIdx.x], s_pool[threadIdx.x]);
}

// Stage 3, one CTA of 64 threads per set: the head on the pooled features.
// Writes pred[4] = (phi, b, slope, theta2) in the original frame and the
// state; with targets, also the loss and dL/d(phi, b).
__global__ void __launch_bounds__(64) k_setnet_head(const __nv_bfloat16 *__restrict__ wb, int B,
                                                    const float *__restrict__ targets, float bweight,
                                                    float *__restrict__ pred, float *__restrict__ state,
                                                    const unsigned long long *__restrict__ pool,
                                                    float *__restrict__ dout)
{
    __shared__ float s_g[H2], s_h3[H3];
    const int set = blockIdx.x;
    if (threadIdx.x < H2) s_g[threadIdx.x] = __uint_as_float((unsigned)(pool[(size_t)set * H2 + threadIdx.x] >> 32));
    __syncthreads();
    if (threadIdx.x < H3) {
        float acc = ld(wb, OFF_B3 + threadIdx.x);
        for (int k = 0; k < H2; ++k) acc = fmaf(ld(wb, OFF_W3 + threadIdx.x * H2 + k), s_g[k], acc);
        s_h3[threadIdx.x] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float *st = state + (size_t)set * STATE;
        const float cx = st[0], cy = st[1], sc = st[2];
        float o[NOUT];
        for (int j = 0; j < NOUT; ++j) {
            float acc = ld(wb, OFF_B4 + j);
            for (int k = 0; k < H3; ++k) acc = fmaf(ld(wb, OFF_W4 + j * H3 + k), s_h3[k], acc);
            o[j] = acc;
        }
        const float phi = o[0], bn = o[1];
        const float slope = tanf(phi);
        const float theta2 = cy + sc * bn - slope * cx;
        float *pr = pred + (size_t)set * 4;
        pr[0] = phi; pr[1] = bn; pr[2] = slope; pr[3] = theta2;
        st[3] = phi; st[4] = bn; st[5] = slope; st[6] = theta2;
        if (targets) {
            const float e0 = phi - targets[2 * set], e1 = bn - targets[2 * set + 1];
            st[7] = (e0 * e0 + bweight * e1 * e1) / (float)B;
            dout[2 * set] = 2.f * e0 / (float)B;
            dout[2 * set + 1] = 2.f * bweight * e1 / (float)B;
        }
    }
}

// The three forward stages on stream st; slices per set so that about two
// CTAs per SM are busy (at most 64, at least 1).
void setnet_forward(const __nv_bfloat16 *wb, float *state, unsigned long long *pool, float *dout, const short *x,
                    const short *y, const long long *off, int B, const float *targets, float bweight, float *pred,
                    cudaStream_t st)
{
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int slices = (2 * (sms > 0 ? sms : 1) + B - 1) / B;
    slices = slices < 1 ? 1 : (slices > 64 ? 64 : slices);
    { StageTimer _t(STAGE_SETNET, st); k_setnet_frame<<<B, 256, 0, st>>>(x, y, off, state, pool); }
    {
        StageTimer _t(STAGE_SETNET, st);
        k_setnet_points<<<dim3(B, slices), 256, 0, st>>>(wb, x, y, off, state, pool);
    }
    {
        StageTimer _t(STAGE_SETNET, st);
        k_setnet_head<<<B, 64, 0, st>>>(wb, B, targets, bweight, pred, state, pool, dout);
    }
}

// Backward: one CTA of 64 threads per set; gradients accumulate into g.
__global__ void __launch_bounds__(64) k_setnet_bwd(const __nv_bfloat16 *__restrict__ wb, const short *__restrict__ x,
                                                   const short *__restrict__ y, const long long *__restrict__ off,
                                                   int B, const float *__restrict__ state,
                                                   const unsigned long long *__restrict__ pool,
                                                   const float *__restrict__ dout, float *__restrict__ g)
{
    __shared__ float s_g[H2], s_h3[H3], s_dz3[H3], s_dg[H2];
    __shared__ float s_dw1[H1 * 2], s_db1[H1];
    const int set = blockIdx.x, c = threadIdx.x;
    if (set >= B) return;
    const unsigned long long pk = pool[(size_t)set * H2 + c];
    s_g[c] = __uint_as_float((unsigned)(pk >> 32));
    s_dw1[2 * c] = 0.f; s_dw1[2 * c + 1] = 0.f; s_db1[c] = 0.f;
    __syncthreads();
    const float d0 = dout[2 * set], d1 = dout[2 * set + 1];
    if (c < H3) {
        float acc = ld(wb, OFF_B3 + c);
        for (int k = 0; k < H2; ++k) acc = fmaf(ld(wb, OFF_W3 + c * H2 + k), s_g[k], acc);
        s_h3[c] = fmaxf(acc, 0.f);
        const float dh3 = ld(wb, OFF_W4 + c) * d0 + ld(wb, OFF_W4 + H3 + c) * d1;
        s_dz3[c] = acc > 0.f ? dh3 : 0.f;
    }
    __syncthreads();
    if (c < H3) {
        atomicAdd(&g[OFF_W4 + c], d0 * s_h3[c]);
        atomicAdd(&g[OFF_W4 + H3 + c], d1 * s_h3[c]);
        atomicAdd(&g[OFF_B3 + c], s_dz3[c]);
        for (int k = 0; k < H2; ++k) atomicAdd(&g[OFF_W3 + c * H2 + k], s_dz3[c] * s_g[k]);
    }
    if (c == 0) { atomicAdd(&g[OFF_B4], d0); atomicAdd(&g[OFF_B4 + 1], d1); }
    {
        float acc = 0.f;
        for (int j = 0; j < H3; ++j) acc = fmaf(ld(wb, OFF_W3 + j * H2 + c), s_dz3[j], acc);
        s_dg[c] = acc;
    }
    __syncthreads();
    // channel c: back through the max-pool to its point, then through the MLP
    const float dz2 = s_g[c] > 0.f ? s_dg[c] : 0.f;
    const float *st = state + (size_t)set * STATE;
    const float cx = st[0], cy = st[1], sc = st[2];
    const long long p = off[set] + (long long)(0xffffffffu - (unsigned)(pk & 0xffffffffu));
    const float inv = 1.0f / sc;
    const float xn = ((float)x[p] - cx) * inv, yn = ((float)y[p] - cy) * inv;
    atomicAdd(&g[OFF_B2 + c], dz2);
    if (dz2 != 0.f) {
        for (int k = 0; k < H1; ++k) {
            float z1 = ld(wb, OFF_B1 + k);
            z1 = fmaf(ld(wb, OFF_W1 + 2 * k), xn, z1);
            z1 = fmaf(ld(wb, OFF_W1 + 2 * k + 1), yn, z1);
            const float h1 = fmaxf(z1, 0.f);
            atomicAdd(&g[OFF_W2 + c * H1 + k], dz2 * h1);
            if (z1 > 0.f) {
                const float t = ld(wb, OFF_W2 + c * H1 + k) * dz2;
                atomicAdd(&s_dw1[2 * k], t * xn);
                atomicAdd(&s_dw1[2 * k + 1], t * yn);
                atomicAdd(&s_db1[k], t);
            }
        }
    }
    __syncthreads();
    atomicAdd(&g[OFF_W1 + 2 * c], s_dw1[2 * c]);
    atomicAdd(&g[OFF_W1 + 2 * c + 1], s_dw1[2 * c + 1]);
    atomicAdd(&g[OFF_B1 + c], s_db1[c]);
}

// Adam on the FP32 master weights; refreshes the BF16-rounded copy.
__global__ void k_adam(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, float *__restrict__ m,
                       float *__restrict__ v, float *__restrict__ g, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float upd = (mk / c1) / (sqrtf(vk / c2) + eps);
    const float nw = w[k] - lr * upd;
    w[k] = nw;
    wb[k] = __float2bfloat16_rn(nw);
    g[k] = 0.f;
}

__global__ void k_round_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) wb[k] = __float2bfloat16_rn(w[k]);
}

__global__ void k_sum_loss(const float *__restrict__ state, int B, float *__restrict__ loss)
{
    float s = 0.f;
    for (int k = threadIdx.x; k < B; k += blockDim.x) s += state[(size_t)k * STATE + 7];
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (threadIdx.x == 0) *loss = s;
}

}  // namespace
}  // namespace lms

using namespace lms;

// {0, n}: the offsets of one set, for the forward pass of a single fit.
__global__ void k_set_offsets(long long *off, long long n)
{
    if (threadIdx.x == 0) { off[0] = 0; off[1] = n; }
}

struct lms_setnet {
    int dev;
    int max_sets;
    long long step;
    float *w, *m, *v, *g;                 // device FP32, NPARAM each
    __nv_bfloat16 *wb;                    // device BF16 copy used by the forward pass
    float *state, *dout, *pred, *loss;    // device, per set
    unsigned long long *pool;             // device, per set x H2
    long long *off1;                      // device, {0, n} for single fits
    short *hx, *hy;                       // device staging of host-buffer fits (65536 points each)
    lms_result *hres;                     // device result of host-buffer fits
    cudaStream_t side;                    // the forward pass of a learned fit runs here ...
    cudaEvent_t ev_fork, ev_join;         // ... beside the branch-and-bound's sampling stage
    // The device part of host-buffer fits (staging to result) as a CUDA graph
    // for one key (n, h, options, workspace generation), captured on `cap` by
    // the second call with that key and replayed by the later ones.
    cudaStream_t cap;
    cudaGraphExec_t hg_exec;
    long long hg_n, hg_h, hg_launches;
    lms_options hg_opt;
    unsigned long long hg_gen;
    int hg_seen;                          // calls with the key so far; negative: capture failed
};

namespace {

int grow_sets(lms_setnet *net, int B)
{
    if (B <= net->max_sets) return LMS_OK;
    cudaDeviceSynchronize();
    if (net->hg_exec) cudaGraphExecDestroy(net->hg_exec);   // it holds the old buffers
    net->hg_exec = nullptr;
    net->hg_seen = 0;
    cudaFree(net->state); cudaFree(net->dout); cudaFree(net->pred); cudaFree(net->pool);
    net->state = nullptr; net->dout = nullptr; net->pred = nullptr; net->pool = nullptr;
    int cap = 64;
    while (cap < B) cap <<= 1;
    if (cudaMalloc(&net->state, sizeof(float) * STATE * cap) != cudaSuccess ||
        cudaMalloc(&net->dout, sizeof(float) * 2 * cap) != cudaSuccess ||
        cudaMalloc(&net->pred, sizeof(float) * 4 * cap) != cudaSuccess ||
        cudaMalloc(&net->pool, sizeof(unsigned long long) * H2 * cap) != cudaSuccess) {
        cudaGetLastError();
        net->max_sets = 0;
        return LMS_ERR_CUDA;
    }
    net->max_sets = cap;
    return LMS_OK;
}

unsigned long long splitmix(unsigned long long &s)
{
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int lms_setnet_create(uint64_t seed, lms_setnet **out)
{
    if (!out) return LMS_ERR_ARG;
    *out = nullptr;
    lms_setnet *net = new lms_setnet();
    memset(net, 0, sizeof(*net));
    cudaGetDevice(&net->dev);
    float **bufs[] = {&net->w, &net->m, &net->v, &net->g};
    for (float **b : bufs) {
        if (cudaMalloc(b, sizeof(float) * NPARAM) != cudaSuccess) { cudaGetLastError(); lms_setnet_destroy(net); return LMS_ERR_CUDA; }
        cudaMemset(*b, 0, sizeof(float) * NPARAM);
    }
    if (cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * NPARAM) != cudaSuccess) {
        cudaGetLastError(); lms_setnet_destroy(net); return LMS_ERR_CUDA;
    }
    if (cudaMalloc(&net->loss, sizeof(float) * 4) != cudaSuccess ||
        cudaMalloc(&net->off1, sizeof(long long) * 2) != cudaSuccess) {
        cudaGetLastError(); lms_setnet_destroy(net); return LMS_ERR_CUDA;
    }
    if (grow_sets(net, 64)) { lms_setnet_destroy(net); return LMS_ERR_CUDA; }
    // He-style uniform init from a SplitMix64 stream; zero biases
    std::vector<float> w(NPARAM, 0.f);
    unsigned long long s = seed;
    auto fill = [&](int off, int count, int fan_in) {
        const float lim = sqrtf(6.0f / (float)fan_in);
        for (int k = 0; k < count; ++k) {
            const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            w[off + k] = (float)((2.0 * u - 1.0) * lim);
        }
    };
    fill(OFF_W1, H1 * 2, 2);
    fill(OFF_W2, H2 * H1, H1);
    fill(OFF_W3, H3 * H2, H2);
    fill(OFF_W4, NOUT * H3, H3);
    cudaMemcpy(net->w, w.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    k_round_bf16<<<(NPARAM + 255) / 256, 256>>>(net->w, net->wb, NPARAM);
    if (cudaDeviceSynchronize() != cudaSuccess) { lms_setnet_destroy(net); return LMS_ERR_CUDA; }
    *out = net;
    return LMS_OK;
}

void lms_setnet_destroy(lms_setnet *net)
{
    if (!net) return;
    cudaFree(net->w); cudaFree(net->wb); cudaFree(net->m); cudaFree(net->v); cudaFree(net->g);
    cudaFree(net->state); cudaFree(net->dout); cudaFree(net->pred); cudaFree(net->pool);
    cudaFree(net->loss); cudaFree(net->off1);
    cudaFree(net->hx); cudaFree(net->hy); cudaFree(net->hres);
    if (net->side) cudaStreamDestroy(net->side);
    if (net->ev_fork) cudaEventDestroy(net->ev_fork);
    if (net->ev_join) cudaEventDestroy(net->ev_join);
    if (net->hg_exec) cudaGraphExecDestroy(net->hg_exec);
    if (net->cap) cudaStreamDestroy(net->cap);
    delete net;
}

int64_t lms_setnet_param_count(void) { return NPARAM; }

int lms_setnet_params(lms_setnet *net, float *host, int64_t count, int32_t set)
{
    if (!net || !host || count != NPARAM) return LMS_ERR_ARG;
    if (set) {
        if (cudaMemcpy(net->w, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return LMS_ERR_CUDA;
        k_round_bf16<<<(NPARAM + 255) / 256, 256>>>(net->w, net->wb, NPARAM);
        return cudaDeviceSynchronize() == cudaSuccess ? LMS_OK : LMS_ERR_CUDA;
    }
    return cudaMemcpy(host, net->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? LMS_OK
                                                                                                   : LMS_ERR_CUDA;
}

int lms_setnet_forward(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets, int64_t B,
                       float *pred, lms_stream_t stream)
{
    if (!net || !x || !y || !offsets || !pred || B < 1) return LMS_ERR_ARG;
    if (grow_sets(net, (int)B)) return LMS_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    setnet_forward(net->wb, net->state, net->pool, net->dout, (const short *)x, (const short *)y,
                   (const long long *)offsets, (int)B, nullptr, 0.f, pred, st);
    return cudaGetLastError() == cudaSuccess ? LMS_OK : LMS_ERR_CUDA;
}

int lms_setnet_backward(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets, int64_t B,
                        const float *targets, float intercept_weight, float *grads, float *loss,
                        lms_stream_t stream)
{
    if (!net || !x || !y || !offsets || !targets || B < 1) return LMS_ERR_ARG;
    if (grow_sets(net, (int)B)) return LMS_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(net->g, 0, sizeof(float) * NPARAM, st);
    setnet_forward(net->wb, net->state, net->pool, net->dout, (const short *)x, (const short *)y,
                   (const long long *)offsets, (int)B, targets, intercept_weight, net->pred, st);
    {
        StageTimer _t(STAGE_SETNET, st);
        k_setnet_bwd<<<(int)B, 64, 0, st>>>(net->wb, (const short *)x, (const short *)y, (const long long *)offsets,
                                            (int)B, net->state, net->pool, net->dout, net->g);
    }
    {
        StageTimer _t(STAGE_SETNET, st);
        k_sum_loss<<<1, 32, 0, st>>>(net->state, (int)B, net->loss);
    }
    if (grads) cudaMemcpyAsync(grads, net->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st);
    if (loss) cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? LMS_OK : LMS_ERR_CUDA;
}

int lms_setnet_train_step(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets, int64_t B,
                          const float *targets, float intercept_weight, float lr, float *loss,
                          lms_stream_t stream)
{
    const int rc = lms_setnet_backward(net, x, y, offsets, B, targets, intercept_weight, nullptr, loss, stream);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    StageTimer _t(STAGE_SETNET, st);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(net->w, net->wb, net->m, net->v, net->g, NPARAM, lr, b1, b2,
                                                1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? LMS_OK : LMS_ERR_CUDA;
}

// File: magic, version, step, NPARAM, then w, m, v (FP32).
int lms_setnet_save(const lms_setnet *net, const char *path)
{
    if (!net || !path) return LMS_ERR_ARG;
    std::vector<float> buf(3 * NPARAM);
    if (cudaDeviceSynchronize() != cudaSuccess) return LMS_ERR_CUDA;
    cudaMemcpy(buf.data(), net->w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + NPARAM, net->m, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + 2 * NPARAM, net->v, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    FILE *f = fopen(path, "wb");
    if (!f) return LMS_ERR_ARG;
    const char magic[8] = {'L', 'M', 'S', 'N', 'E', 'T', '0', '1'};
    const long long hdr[2] = {net->step, NPARAM};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(long long), 2, f) == 2 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? LMS_OK : LMS_ERR_ARG;
}

int lms_setnet_load(lms_setnet *net, const char *path)
{
    if (!net || !path) return LMS_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return LMS_ERR_ARG;
    char magic[8];
    long long hdr[2];
    std::vector<float> buf(3 * NPARAM);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "LMSNET01", 8) == 0 &&
              fread(hdr, sizeof(long long), 2, f) == 2 && hdr[1] == NPARAM &&
              fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return LMS_ERR_ARG;
    net->step = hdr[0];
    cudaMemcpy(net->w, buf.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    cudaMemcpy(net->m, buf.data() + NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    cudaMemcpy(net->v, buf.data() + 2 * NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    k_round_bf16<<<(NPARAM + 255) / 256, 256>>>(net->w, net->wb, NPARAM);
    return cudaDeviceSynchronize() == cudaSuccess ? LMS_OK : LMS_ERR_CUDA;
}

int lms_fit_learned(lms_setnet *net, const void *x, const void *y, int64_t n, int64_t h, const lms_options *opt,
                    lms_result *out, lms_bnb_stats *stats, lms_stream_t stream)
{
    // every argument is checked before the forward pass is queued on the
    // side stream
    if (!net || check_bnb_args(x, y, n, h, opt, out)) return LMS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!net->side) {
        if (cudaStreamCreateWithFlags(&net->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return LMS_ERR_CUDA;
        }
    }
    // the forward pass runs on the net's side stream, forked from and joined
    // back to `stream`: the branch-and-bound samples and sorts pair slopes
    // meanwhile and waits for the prediction only where it picks its seeds
    if (cudaEventRecord(net->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(net->side, net->ev_fork, 0) != cudaSuccess)
        return LMS_ERR_CUDA;
    {
        StageTimer _t(STAGE_SETNET, net->side);
        k_set_offsets<<<1, 32, 0, net->side>>>(net->off1, n);
    }
    int rc = lms_setnet_forward(net, (const int16_t *)x, (const int16_t *)y, (const int64_t *)net->off1, 1,
                                net->pred, reinterpret_cast<lms_stream_t>(net->side));
    if (rc) return rc;
    if (cudaEventRecord(net->ev_join, net->side) != cudaSuccess) return LMS_ERR_CUDA;
    // pred[2] is the predicted slope in the original frame
    return fit_bnb_after(x, y, n, h, net->pred + 2, opt, out, stats, st, net->ev_join);
}

}  // extern "C"

namespace {

// The device part of a host-buffer fit (points already staged in hx, hy;
// result into hres), by replaying the graph cached for its key.  The first
// call with a key returns false (the caller fits directly, which also grows
// every buffer the fit needs); the second captures the fit on the net's own
// stream (any stream the caller passes, the legacy default stream included,
// can then launch it) and replays it.  Returns false also for a key whose
// capture failed; otherwise rc holds the launch status.
bool replay_host_fit(lms_setnet *net, int64_t n, int64_t h, const lms_options *opt, cudaStream_t st, int &rc)
{
    lms_options o;
    memset(&o, 0, sizeof o);
    if (opt) memcpy(&o, opt, sizeof o);
    const unsigned long long gen = workspace_generation();
    if (net->hg_n != n || net->hg_h != h || net->hg_gen != gen || memcmp(&net->hg_opt, &o, sizeof o) != 0) {
        if (net->hg_exec) cudaGraphExecDestroy(net->hg_exec);
        net->hg_exec = nullptr;
        net->hg_n = n;
        net->hg_h = h;
        net->hg_gen = gen;
        memcpy(&net->hg_opt, &o, sizeof o);
        net->hg_seen = 0;
    }
    if (!net->hg_exec) {
        if (net->hg_seen < 1) {
            if (net->hg_seen == 0) net->hg_seen = 1;
            return false;
        }
        if (!net->cap && cudaStreamCreateWithFlags(&net->cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            net->cap = nullptr;
            net->hg_seen = -1;
            return false;
        }
        const long long l0 = lms_launch_count();
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        if (cudaStreamBeginCapture(net->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int frc = lms_fit_learned(net, net->hx, net->hy, n, h, opt, net->hres, nullptr,
                                            reinterpret_cast<lms_stream_t>(net->cap));
            const cudaError_t ce = cudaStreamEndCapture(net->cap, &g);
            if (frc == LMS_OK && ce == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess)
                ex = nullptr;
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (!ex) {
            net->hg_seen = -1;
            return false;
        }
        net->hg_exec = ex;
        net->hg_launches = lms_launch_count() - l0;
    }
    if (cudaGraphLaunch(net->hg_exec, st) != cudaSuccess) {
        cudaGetLastError();
        rc = LMS_ERR_CUDA;
        return true;
    }
    add_launches(net->hg_launches);
    rc = LMS_OK;
    return true;
}

}  // namespace

extern "C" {

int lms_fit_learned_host(lms_setnet *net, const void *x, const void *y, int64_t n, int64_t h,
                         const lms_options *opt, lms_result *out, lms_bnb_stats *stats, lms_stream_t stream)
{
    if (!net || check_bnb_args(x, y, n, h, opt, out)) return LMS_ERR_ARG;
    if (!net->hx) {
        if (cudaMalloc(&net->hx, sizeof(short) * 65536) != cudaSuccess ||
            cudaMalloc(&net->hy, sizeof(short) * 65536) != cudaSuccess ||
            cudaMalloc(&net->hres, sizeof(lms_result)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(net->hx); cudaFree(net->hy); cudaFree(net->hres);
            net->hx = net->hy = nullptr;
            net->hres = nullptr;
            return LMS_ERR_CUDA;
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(net->hx, x, sizeof(short) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(net->hy, y, sizeof(short) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    int rc = LMS_OK;
    if (!stats && !profiling_on() && replay_host_fit(net, n, h, opt, st, rc)) {
        if (rc) return rc;
    } else {
        rc = lms_fit_learned(net, net->hx, net->hy, n, h, opt, net->hres, stats, stream);
        if (rc) return rc;
    }
    if (cudaMemcpyAsync(out, net->hres, sizeof(lms_result), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LMS_ERR_CUDA;
    return LMS_OK;
}

}  // extern "C"
