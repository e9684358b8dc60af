// batched.cu -- many exact LMS fits of uneven size in one call.
//
// A plan is made once from the host offsets of the point sets: sets with at
// most `plain_max` points go to one persistent plain kernel whose work items
// are (set, run of consecutive slopes) chunks, grouped by size class so each
// class sorts in registers of the right width (E = 2, 4, 8 keys per lane for
// n <= 64, 128, 256); larger sets each get the exact sweep pipeline, spread
// over a few internal streams with their own workspaces.  lms_fit_batched
// then only enqueues kernels: no allocation and no host synchronisation, so
// a whole batch can be captured into one CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr int CHUNK = 64;   // slopes per work item of the plain kernel
constexpr int BATCH_BNB_MIN_N = 512;   // default size from which a set takes the branch-and-bound

template <typename K>
__device__ __forceinline__ void cxk(K &a, K &b)
{
    K lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Warp bitonic sort of 32*E keys (blocked index lane*E + r, see plain.cu).
template <int E, typename K>
__device__ __forceinline__ void wsort(K (&v)[E], int lane)
{
    constexpr int P = 32 * E;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
        if (k <= E) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int q = r ^ (k - 1);
                if (q > r) cxk(v[r], v[q]);
            }
        } else {
            const int lm = k / E - 1;
            const bool lower = (lane & (k / (2 * E))) == 0;
            K tmp[E];
#pragma unroll
            for (int r = 0; r < E; ++r) tmp[r] = __shfl_xor_sync(FULL, v[E - 1 - r], lm);
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = lower ? min(v[r], tmp[r]) : max(v[r], tmp[r]);
        }
#pragma unroll
        for (int j = k / 4; j >= 1; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int q = r ^ j;
                    if (q > r) cxk(v[r], v[q]);
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

// One warp per chunk of at most CHUNK consecutive slopes of one set.
// chunk_pre[i] = chunks before class-set i; sets[i] = global set index.
template <int E>
__global__ void __launch_bounds__(256) k_plain_batched(const short *__restrict__ x, const short *__restrict__ y,
                                                       const long long *__restrict__ off,
                                                       const int *__restrict__ hvec,
                                                       const int *__restrict__ sets, int nsets,
                                                       const long long *__restrict__ chunk_pre,
                                                       Cand *__restrict__ outc)
{
    __shared__ long long s_buf[8][32 * E];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nchunks = chunk_pre[nsets];
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp; c < nchunks;
         c += (long long)gridDim.x * (blockDim.x >> 5)) {
        int lo = 0, hi = nsets;
        while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (chunk_pre[mid] <= c) lo = mid; else hi = mid; }
        const int si = lo;
        const long long base = off[sets[si]];
        const int n = (int)(off[sets[si] + 1] - base);
        const int h = hvec[sets[si]];
        const long long npairs = (long long)n * (n - 1) / 2;
        const long long g0 = (c - chunk_pre[si]) * CHUNK, g1 = min(npairs, g0 + CHUNK);
        int P[E];
        int xmin = 1 << 30, xmax = -(1 << 30), ymin = 1 << 30, ymax = -(1 << 30);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = r * 32 + lane;
            P[r] = k < n ? pack_xy(x[base + k], y[base + k]) : 0;
            if (k < n) {
                xmin = min(xmin, px(P[r])); xmax = max(xmax, px(P[r]));
                ymin = min(ymin, py(P[r])); ymax = max(ymax, py(P[r]));
            }
        }
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            xmin = min(xmin, __shfl_xor_sync(FULL, xmin, s)); xmax = max(xmax, __shfl_xor_sync(FULL, xmax, s));
            ymin = min(ymin, __shfl_xor_sync(FULL, ymin, s)); ymax = max(ymax, __shfl_xor_sync(FULL, ymax, s));
        }
        const long long bound = (long long)max(-ymin, ymax) * (xmax - xmin) +
                                (long long)max(-xmin, xmax) * (ymax - ymin);
        const bool fits32 = bound < 0x7fffffffLL;
        Cand best = cand_empty();
        for (long long g = g0; g < g1; ++g) {
            int i, j;
            pair_decode(g, i, j);
            const int pi = pack_xy(x[base + i], y[base + i]), pj = pack_xy(x[base + j], y[base + j]);
            int dy, dx;
            if (!pair_slope(pi, pj, dy, dx)) continue;
            long long bw = 0x7fffffffffffffffLL;
            int ba = 0x7fffffff;
            if (fits32) {
                int v[E];
#pragma unroll
                for (int r = 0; r < E; ++r)
                    v[r] = (r * 32 + lane < n) ? py(P[r]) * dx - px(P[r]) * dy : 0x7fffffff;
                wsort<E, int>(v, lane);
#pragma unroll
                for (int r = 0; r < E; ++r) s_buf[warp][lane * E + r] = v[r];
            } else {
                long long v[E];
#pragma unroll
                for (int r = 0; r < E; ++r)
                    v[r] = (r * 32 + lane < n) ? (long long)py(P[r]) * dx - (long long)px(P[r]) * dy
                                               : 0x7fffffffffffffffLL;
                wsort<E, long long>(v, lane);
#pragma unroll
                for (int r = 0; r < E; ++r) s_buf[warp][lane * E + r] = v[r];
            }
            __syncwarp();
            for (int a = lane; a + h - 1 < n; a += 32) {
                const long long wd = s_buf[warp][a + h - 1] - s_buf[warp][a];
                if (wd < bw) { bw = wd; ba = a; }
            }
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const long long ow = __shfl_xor_sync(FULL, bw, s);
                const int oa = __shfl_xor_sync(FULL, ba, s);
                if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
            }
            Cand cd;
            cd.w = bw; cd.t = s_buf[warp][ba] + s_buf[warp][ba + h - 1]; cd.dy = dy; cd.dx = dx; cd.i = i; cd.j = j;
            __syncwarp();
            if (cand_better(cd, best)) best = cd;
        }
        if (lane == 0) outc[c] = best;
    }
}

// Per set of a size class: the best record over its chunks (vertical sets:
// the window at slope 0), then the final translation.
__global__ void k_plain_batched_reduce(const short *__restrict__ x, const short *__restrict__ y,
                                       const long long *__restrict__ off, const int *__restrict__ hvec,
                                       const int *__restrict__ sets, int nsets,
                                       const long long *__restrict__ chunk_pre, const Cand *__restrict__ outc,
                                       Cand *__restrict__ best_out)
{
    const int lane = threadIdx.x & 31;
    const int si = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (si >= nsets) return;
    Cand best = cand_empty();
    for (long long c = chunk_pre[si] + lane; c < chunk_pre[si + 1]; c += 32)
        if (cand_better(outc[c], best)) best = outc[c];
    best = warp_best(best);
    if (best.dx == 0) {
        // every x equal (or fewer than two points): the window at slope 0
        __shared__ long long s_y[8][256];
        const int w = threadIdx.x >> 5;
        const long long base = off[sets[si]];
        const int n = (int)(off[sets[si] + 1] - base), h = hvec[sets[si]];
        long long v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = (r * 32 + lane < n) ? (long long)y[base + r * 32 + lane] : 0x7fffffffffffffffLL;
        wsort<8, long long>(v, lane);
#pragma unroll
        for (int r = 0; r < 8; ++r) s_y[w][lane * 8 + r] = v[r];
        __syncwarp();
        long long bw = 0x7fffffffffffffffLL;
        int ba = 0x7fffffff;
        for (int q = lane; q + h - 1 < n; q += 32) {
            const long long wd = s_y[w][q + h - 1] - s_y[w][q];
            if (wd < bw) { bw = wd; ba = q; }
        }
        for (int s = 16; s >= 1; s >>= 1) {
            const long long ow = __shfl_xor_sync(FULL, bw, s);
            const int oa = __shfl_xor_sync(FULL, ba, s);
            if (ow < bw || (ow == bw && oa < ba)) { bw = ow; ba = oa; }
        }
        best.w = bw; best.t = s_y[w][ba] + s_y[w][ba + h - 1];
        best.dy = 0; best.dx = 1; best.i = -1; best.j = -1;
    }
    if (lane == 0) best_out[si] = best;
}

__device__ __forceinline__ long long gcd_ll(long long a, long long b)
{
    while (b) { long long r = a % b; a = b; b = r; }
    return a;
}

// Translate per-set winners into lms_result records at their set indices.
__global__ void k_batched_finish(const Cand *__restrict__ best, const int *__restrict__ sets, int nsets,
                                 lms_result *__restrict__ out)
{
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= nsets) return;
    const Cand b = best[si];
    lms_result r;
    r.algorithm = LMS_ALGO_PLAIN;
    const long long dx = b.dx, dy = b.dy;
    long long g = gcd_ll(dy < 0 ? -dy : dy, dx);
    if (g <= 0) g = 1;
    r.s_num = dy / g; r.s_den = dx / g;
    r.w_num = b.w / g; r.w_den = r.s_den;
    r.t_num = b.t / g; r.t_den = 2 * r.s_den;
    r.theta1 = __ddiv_rn((double)r.s_num, (double)r.s_den);
    r.theta2 = __ddiv_rn((double)r.t_num, (double)r.t_den);
    const double half = __ddiv_rn((double)r.w_num, (double)(2 * r.w_den));
    r.med_sq = __dmul_rn(half, half);
    r.i = b.i; r.j = b.j;
    r.status = b.i < 0 ? LMS_ERR_VERTICAL : LMS_OK;
    out[sets[si]] = r;
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lms

using namespace lms;

struct lms_batch_plan {
    int dev = 0;
    int64_t B = 0;
    int plain_max = 256;
    int bnb_min = 0;                    // sets of at least this many points take the branch-and-bound
    // plain classes (E = 2, 4, 8)
    struct Cls {
        int E = 0;
        int nsets = 0;
        long long nchunks = 0;
        int *sets = nullptr;            // device
        long long *chunk_pre = nullptr; // device
        Cand *outc = nullptr;           // device, one record per chunk
        Cand *best = nullptr;           // device
    } cls[3];
    int *hvec = nullptr;                // device, per set
    // sweep sets
    std::vector<long long> off_host;
    std::vector<int> sweep_sets;        // global indices, assigned to streams
    std::vector<int> stream_of;
    int nstreams = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_done;
    cudaEvent_t ev_start = nullptr;
    std::vector<void *> ws;             // per stream sweep workspace
    std::vector<int> hval;              // host copy of h per set
    size_t bytes = 0;
    void *mem = nullptr;                // one allocation for the plain tables
};

extern "C" {

int lms_batch_plan_create(const int64_t *offsets_host, int64_t B, const int32_t *h_host, int32_t plain_max_n,
                          int32_t nstreams, lms_batch_plan **out)
{
    return lms_batch_plan_create_ex(offsets_host, B, h_host, plain_max_n, nstreams, 0, out);
}

int lms_batch_plan_create_ex(const int64_t *offsets_host, int64_t B, const int32_t *h_host, int32_t plain_max_n,
                             int32_t nstreams, int32_t bnb_min_n, lms_batch_plan **out)
{
    if (!offsets_host || B < 1 || !out) return LMS_ERR_ARG;
    *out = nullptr;
    for (int64_t i = 0; i < B; ++i) {
        const int64_t n = offsets_host[i + 1] - offsets_host[i];
        if (n < 2 || n > 32768) return LMS_ERR_ARG;
    }
    lms_batch_plan *p = new lms_batch_plan();
    cudaGetDevice(&p->dev);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev);
    p->B = B;
    p->plain_max = plain_max_n > 0 ? std::min(plain_max_n, 256) : 256;
    // sets from this size on take the branch-and-bound (its fixed cost, a few
    // hundred microseconds of seeds and bounds, pays off once the sweep of every
    // slope costs more); negative: never
    p->bnb_min = bnb_min_n > 0 ? std::max(bnb_min_n, 257) : (bnb_min_n < 0 ? 0x7fffffff : BATCH_BNB_MIN_N);
    p->off_host.assign(offsets_host, offsets_host + B + 1);
    p->hval.resize(B);
    for (int64_t i = 0; i < B; ++i) {
        const int64_t n = offsets_host[i + 1] - offsets_host[i];
        int h = h_host ? h_host[i] : 0;
        if (h == 0) h = (int)(n / 2 + 1);
        if (h < 1 || h > n) { delete p; return LMS_ERR_ARG; }
        p->hval[i] = h;
    }
    // classes
    std::vector<int> members[3];
    for (int64_t i = 0; i < B; ++i) {
        const int64_t n = offsets_host[i + 1] - offsets_host[i];
        if (n <= p->plain_max) members[n <= 64 ? 0 : (n <= 128 ? 1 : 2)].push_back((int)i);
        else p->sweep_sets.push_back((int)i);
    }
    size_t bytes = a256(sizeof(int) * B);
    std::vector<std::vector<long long>> pres(3);
    for (int c = 0; c < 3; ++c) {
        p->cls[c].E = 2 << c;
        p->cls[c].nsets = (int)members[c].size();
        auto &pre = pres[c];
        pre.assign(members[c].size() + 1, 0);
        for (size_t k = 0; k < members[c].size(); ++k) {
            const long long n = offsets_host[members[c][k] + 1] - offsets_host[members[c][k]];
            pre[k + 1] = pre[k] + (n * (n - 1) / 2 + CHUNK - 1) / CHUNK;
        }
        p->cls[c].nchunks = pre.back();
        bytes += a256(sizeof(int) * members[c].size()) + a256(sizeof(long long) * pre.size()) +
                 a256(sizeof(Cand) * (size_t)std::max<long long>(1, p->cls[c].nchunks)) +
                 a256(sizeof(Cand) * std::max<size_t>(1, members[c].size()));
    }
    if (cudaMalloc(&p->mem, bytes) != cudaSuccess) { cudaGetLastError(); delete p; return LMS_ERR_CUDA; }
    p->bytes = bytes;
    unsigned char *q = static_cast<unsigned char *>(p->mem);
    auto take = [&](size_t b) { void *r = q; q += a256(b); return r; };
    p->hvec = (int *)take(sizeof(int) * B);
    cudaMemcpy(p->hvec, p->hval.data(), sizeof(int) * B, cudaMemcpyHostToDevice);
    for (int c = 0; c < 3; ++c) {
        auto &C = p->cls[c];
        C.sets = (int *)take(sizeof(int) * members[c].size());
        C.chunk_pre = (long long *)take(sizeof(long long) * pres[c].size());
        C.outc = (Cand *)take(sizeof(Cand) * (size_t)std::max<long long>(1, C.nchunks));
        C.best = (Cand *)take(sizeof(Cand) * std::max<size_t>(1, members[c].size()));
        if (!members[c].empty())
            cudaMemcpy(C.sets, members[c].data(), sizeof(int) * members[c].size(), cudaMemcpyHostToDevice);
        cudaMemcpy(C.chunk_pre, pres[c].data(), sizeof(long long) * pres[c].size(), cudaMemcpyHostToDevice);
    }
    // sweep sets: largest first onto the least loaded stream
    int ns = nstreams > 0 ? nstreams : 8;
    if (p->sweep_sets.empty()) ns = 0;
    ns = std::min<int>(ns, (int)p->sweep_sets.size());
    p->nstreams = ns;
    std::sort(p->sweep_sets.begin(), p->sweep_sets.end(), [&](int a, int b) {
        return offsets_host[a + 1] - offsets_host[a] > offsets_host[b + 1] - offsets_host[b];
    });
    std::vector<double> load(ns, 0.0);
    std::vector<size_t> need(ns, 0);
    p->stream_of.resize(p->sweep_sets.size());
    for (size_t k = 0; k < p->sweep_sets.size(); ++k) {
        const double n = (double)(offsets_host[p->sweep_sets[k] + 1] - offsets_host[p->sweep_sets[k]]);
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p->stream_of[k] = s;
        load[s] += n * n;
        SweepPlan sp;
        sweep_plan_configure(sp, (int)n, p->hval[p->sweep_sets[k]], sms, 0, 0, true);
        size_t b = sweep_plan_bytes(sp);
        if (n >= p->bnb_min) b = a256(b) + bnb_extra_bytes((int)n, sms);
        need[s] = std::max(need[s], b);
    }
    p->streams.resize(ns);
    p->ev_done.resize(ns);
    p->ws.assign(ns, nullptr);
    cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    for (int s = 0; s < ns; ++s) {
        cudaStreamCreateWithFlags(&p->streams[s], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&p->ev_done[s], cudaEventDisableTiming);
        const size_t b = need[s];
        if (cudaMalloc(&p->ws[s], b) != cudaSuccess) { cudaGetLastError(); lms_batch_plan_destroy(p); return LMS_ERR_CUDA; }
        p->bytes += b;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { lms_batch_plan_destroy(p); return LMS_ERR_CUDA; }
    *out = p;
    return LMS_OK;
}

int lms_batch_plan_destroy(lms_batch_plan *p)
{
    if (!p) return LMS_OK;
    cudaDeviceSynchronize();
    for (void *w : p->ws) cudaFree(w);
    for (cudaStream_t s : p->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : p->ev_done) cudaEventDestroy(e);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    cudaFree(p->mem);
    delete p;
    return LMS_OK;
}

size_t lms_batch_plan_bytes(const lms_batch_plan *p) { return p ? p->bytes : 0; }

int lms_fit_batched(lms_batch_plan *p, const void *xv, const void *yv, const int64_t *offsets_dev, lms_result *out,
                    lms_stream_t stream)
{
    if (!p || !xv || !yv || !offsets_dev || !out) return LMS_ERR_ARG;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->dev) return LMS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const short *x = static_cast<const short *>(xv), *y = static_cast<const short *>(yv);
    const long long *off = reinterpret_cast<const long long *>(offsets_dev);
    cudaGetLastError();
    // fork the sweep streams off the caller's stream
    if (p->nstreams > 0) {
        cudaEventRecord(p->ev_start, st);
        for (int s = 0; s < p->nstreams; ++s) cudaStreamWaitEvent(p->streams[s], p->ev_start, 0);
    }
    // plain classes on the caller's stream
    for (int c = 0; c < 3; ++c) {
        auto &C = p->cls[c];
        if (C.nsets == 0) continue;
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long blocks = std::min<long long>((C.nchunks + 7) / 8, (long long)sms * 8);
        if (C.nchunks > 0) {
            StageTimer _t(STAGE_PLAIN, st);
            switch (C.E) {
                case 2: k_plain_batched<2><<<(int)std::max(1LL, blocks), 256, 0, st>>>(x, y, off, p->hvec, C.sets, C.nsets, C.chunk_pre, C.outc); break;
                case 4: k_plain_batched<4><<<(int)std::max(1LL, blocks), 256, 0, st>>>(x, y, off, p->hvec, C.sets, C.nsets, C.chunk_pre, C.outc); break;
                default: k_plain_batched<8><<<(int)std::max(1LL, blocks), 256, 0, st>>>(x, y, off, p->hvec, C.sets, C.nsets, C.chunk_pre, C.outc); break;
            }
        }
        {
            StageTimer _t(STAGE_ARGMIN, st);
            k_plain_batched_reduce<<<(C.nsets + 7) / 8, 256, 0, st>>>(x, y, off, p->hvec, C.sets, C.nsets, C.chunk_pre,
                                                                      C.outc, C.best);
        }
        {
            StageTimer _t(STAGE_ARGMIN, st);
            k_batched_finish<<<(C.nsets + 127) / 128, 128, 0, st>>>(C.best, C.sets, C.nsets, out);
        }
    }
    // sweep sets on their streams
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bool failed = false;
    for (size_t k = 0; k < p->sweep_sets.size() && !failed; ++k) {
        const int i = p->sweep_sets[k];
        const int s = p->stream_of[k];
        const long long a = p->off_host[i];
        const int n = (int)(p->off_host[i + 1] - a);
        SweepPlan sp;
        sweep_plan_configure(sp, n, p->hval[i], sms, 0, 0, true);
        sweep_plan_carve(sp, p->ws[s]);
        if (n >= p->bnb_min) {
            // asynchronous without statistics: nothing waits on the host
            unsigned char *extra = static_cast<unsigned char *>(p->ws[s]) + a256(sweep_plan_bytes(sp));
            failed = run_bnb(sp, x + a, y + a, nullptr, 0, out + i, nullptr, extra, sms, p->streams[s]) != LMS_OK;
        } else {
            failed = launch_sweep(sp, x + a, y + a, p->streams[s]) != cudaSuccess ||
                     launch_argmin(sp.cands, sp.W + sp.G, out + i, LMS_ALGO_SWEEP, sp.meta + 3, p->streams[s]) !=
                         cudaSuccess;
        }
    }
    // join every forked stream back to the caller's, also after a failed
    // launch, so the caller's stream stays ordered after all queued work
    for (int s = 0; s < p->nstreams; ++s) {
        cudaEventRecord(p->ev_done[s], p->streams[s]);
        cudaStreamWaitEvent(st, p->ev_done[s], 0);
    }
    return (cudaGetLastError() == cudaSuccess && !failed) ? LMS_OK : LMS_ERR_CUDA;
}

}  // extern "C"
