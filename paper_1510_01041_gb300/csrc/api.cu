// api.cu -- the C ABI declared in include/lms.h.
//
// Argument checking, algorithm choice, workspace management and launch
// sequencing.  Every step of a fit runs in the kernels of this library; the
// host only enqueues work on the caller's stream.
#include <cuda_runtime.h>

#include <mutex>
#include <string.h>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

struct DeviceWs {
    void *own = nullptr;       // internal buffer
    size_t own_bytes = 0;
    void *ext = nullptr;       // caller-installed buffer
    size_t ext_bytes = 0;
    unsigned long long gen = 0;   // bumped whenever the buffer in use may change
};

constexpr int MAX_DEV = 64;
std::mutex g_mu;
DeviceWs g_ws[MAX_DEV];

int current_device(int &dev)
{
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return LMS_ERR_CUDA;
    return LMS_OK;
}

int sm_count(int dev)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// Returns a device buffer of at least `bytes`; grows the internal one when
// needed (not allowed while the stream is being captured).
int workspace(size_t bytes, cudaStream_t st, void **out)
{
    int dev;
    if (current_device(dev)) return LMS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceWs &w = g_ws[dev];
    if (w.ext) {
        if (w.ext_bytes < bytes) return LMS_ERR_WORKSPACE;
        *out = w.ext;
        return LMS_OK;
    }
    if (w.own_bytes < bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return LMS_ERR_WORKSPACE;
        if (w.own) {
            cudaDeviceSynchronize();
            cudaFree(w.own);
            w.own = nullptr;
            w.own_bytes = 0;
        }
        size_t grow = bytes + bytes / 8 + (1u << 20);
        ++w.gen;
        if (cudaMalloc(&w.own, grow) != cudaSuccess) {
            cudaGetLastError();
            w.own = nullptr;
            return LMS_ERR_CUDA;
        }
        w.own_bytes = grow;
    }
    *out = w.own;
    return LMS_OK;
}

struct Choice {
    int algo;
    SweepPlan sweep;
    int plain_warps;
    int sms;
    size_t bytes;
    size_t bnb_off;   // offset of the branch-and-bound scratch
    size_t f32_off;   // offset of the float32 sweep scratch
};

int plain_warps_for(int n, int sms)
{
    const long long npairs = (long long)n * (n - 1) / 2;
    long long w = (long long)sms * 32;           // 4 CTAs x 8 warps per SM
    long long need = (npairs + 3) / 4;          // at least ~4 slopes per warp
    if (need < w) w = need;
    w = (w + 7) / 8 * 8;
    return (int)(w < 8 ? 8 : w);
}

int choose(int n, int h, int dtype, const lms_options *opt, int dev, Choice &c)
{
    const int algo_req = opt ? opt->algorithm : LMS_ALGO_AUTO;
    int algo = algo_req;
    // the per-slope warp kernel wins up to about 512 points (0.29 ms against
    // 0.47 ms for the sweep at n = 512 on a GB300), the sweep above
    if (algo == LMS_ALGO_AUTO) algo = (n <= 512 && dtype == LMS_I16) ? LMS_ALGO_PLAIN : LMS_ALGO_SWEEP;
    if (dtype == LMS_F32 && algo != LMS_ALGO_SWEEP) return LMS_ERR_UNSUPPORTED;
    const int sms = sm_count(dev);
    c.algo = algo;
    c.sms = sms;
    c.bnb_off = 0;
    c.f32_off = 0;
    if (algo == LMS_ALGO_PLAIN) {
        if (n > 1024) return LMS_ERR_UNSUPPORTED;
        c.plain_warps = plain_warps_for(n, sms);
        c.bytes = ((size_t)c.plain_warps * sizeof(Cand) + 255) / 256 * 256;
    } else if (algo == LMS_ALGO_PAPER) {
        if (n > 1024) return LMS_ERR_UNSUPPORTED;
        c.bytes = paper_bytes(n);
    } else if (algo == LMS_ALGO_SWEEP || algo == LMS_ALGO_BNB) {
        if (dtype == LMS_F32 && n > 32768) return LMS_ERR_UNSUPPORTED;
        sweep_plan_configure(c.sweep, n, h, sms, opt ? opt->sweepers : 0, opt ? opt->buckets : 0);
        c.bytes = sweep_plan_bytes(c.sweep);
        if (algo == LMS_ALGO_BNB) {
            c.bnb_off = c.bytes;
            c.bytes += bnb_extra_bytes(n, sms);
        }
        if (dtype == LMS_F32) {
            c.f32_off = c.bytes;
            c.bytes += sweep_f32_extra_bytes(n, c.sweep.W);
        }
    } else {
        return LMS_ERR_ARG;
    }
    c.bytes += 256;   // result staging for host-pointer calls
    return LMS_OK;
}

int check_args(const void *x, const void *y, int64_t n, int64_t &h, int32_t dtype, const lms_options *opt,
               const void *out)
{
    if (!x || !y || !out) return LMS_ERR_ARG;
    if (n < 2 || n > 65536) return LMS_ERR_ARG;
    if (h == 0) h = n / 2 + 1;
    if (h < 1 || h > n) return LMS_ERR_ARG;
    if (dtype != LMS_I16 && dtype != LMS_F32) return LMS_ERR_ARG;
    if (opt) {
        if (opt->algorithm < LMS_ALGO_AUTO || opt->algorithm > LMS_ALGO_PAPER) return LMS_ERR_ARG;
        if (opt->sweepers < 0 || opt->buckets < 0) return LMS_ERR_ARG;
        if (opt->seed_mode < 0 || opt->seed_mode > 1) return LMS_ERR_ARG;
        for (int k = 0; k < 4; ++k)
            if (opt->reserved[k]) return LMS_ERR_ARG;
    }
    return LMS_OK;
}

// Enqueue one fit on device buffers.
int run_fit(const void *x, const void *y, int n, int h, int dtype, const lms_options *opt, lms_result *out,
            cudaStream_t st, void *ws_in, const Choice &c)
{
    cudaGetLastError();
    if (c.algo == LMS_ALGO_PLAIN) {
        Cand *cands = static_cast<Cand *>(ws_in);
        if (launch_plain((const short *)x, (const short *)y, n, h, cands, c.plain_warps, st) != cudaSuccess)
            return LMS_ERR_CUDA;
        if (launch_argmin(cands, c.plain_warps, out, LMS_ALGO_PLAIN, nullptr, st) != cudaSuccess)
            return LMS_ERR_CUDA;
        return LMS_OK;
    }
    if (c.algo == LMS_ALGO_PAPER) {
        Cand *cands = nullptr;
        long long count = 0;
        if (launch_paper((const short *)x, (const short *)y, n, h, ws_in, &cands, &count, st) != cudaSuccess)
            return LMS_ERR_CUDA;
        if (launch_argmin(cands, (int)count, out, LMS_ALGO_PAPER, nullptr, st) != cudaSuccess) return LMS_ERR_CUDA;
        return LMS_OK;
    }
    SweepPlan p = c.sweep;
    sweep_plan_carve(p, ws_in);
    if (dtype == LMS_F32)
        return launch_sweep_f32_fit(p, (const float *)x, (const float *)y,
                                    static_cast<unsigned char *>(ws_in) + c.f32_off, out, st) == cudaSuccess
                   ? LMS_OK
                   : LMS_ERR_CUDA;
    if (c.algo == LMS_ALGO_BNB)
        return run_bnb(p, (const short *)x, (const short *)y, nullptr, opt ? opt->seed_mode : 0, out, nullptr,
                       static_cast<unsigned char *>(ws_in) + c.bnb_off, c.sms, st);
    if (launch_sweep(p, (const short *)x, (const short *)y, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (launch_argmin(p.cands, p.W + p.G, out, LMS_ALGO_SWEEP, p.meta + 3, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    return LMS_OK;
}

}  // namespace

unsigned long long workspace_generation()
{
    int dev;
    if (current_device(dev)) return ~0ull;
    std::lock_guard<std::mutex> lock(g_mu);
    return g_ws[dev].gen;
}

int check_bnb_args(const void *x, const void *y, int64_t n, int64_t h, const lms_options *opt, const void *out)
{
    lms_options o = opt ? *opt : lms_options{};
    o.algorithm = LMS_ALGO_BNB;
    return check_args(x, y, n, h, LMS_I16, &o, out);
}

int fit_bnb_after(const void *x, const void *y, int64_t n, int64_t h, const float *seed_slope, const lms_options *opt,
                  lms_result *out, lms_bnb_stats *stats, cudaStream_t st, cudaEvent_t pred_ready)
{
    lms_options o = opt ? *opt : lms_options{};
    o.algorithm = LMS_ALGO_BNB;
    int rc = check_args(x, y, n, h, LMS_I16, &o, out);
    if (rc) return rc;
    int dev;
    if (current_device(dev)) return LMS_ERR_CUDA;
    Choice c;
    rc = choose((int)n, (int)h, LMS_I16, &o, dev, c);
    if (rc) return rc;
    void *ws = nullptr;
    rc = workspace(c.bytes, st, &ws);
    if (rc) return rc;
    SweepPlan p = c.sweep;
    sweep_plan_carve(p, ws);
    cudaGetLastError();
    return run_bnb(p, (const short *)x, (const short *)y, seed_slope, o.seed_mode, out, stats,
                   static_cast<unsigned char *>(ws) + c.bnb_off, c.sms, st, pred_ready);
}

}  // namespace lms

using namespace lms;

extern "C" {

int lms_fit(const void *x, const void *y, int64_t n, int64_t h, int32_t dtype, const lms_options *opt,
            lms_result *out, lms_stream_t stream)
{
    int rc = check_args(x, y, n, h, dtype, opt, out);
    if (rc) return rc;
    int dev;
    if (current_device(dev)) return LMS_ERR_CUDA;
    Choice c;
    rc = choose((int)n, (int)h, dtype, opt, dev, c);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    rc = workspace(c.bytes, st, &ws);
    if (rc) return rc;
    return run_fit(x, y, (int)n, (int)h, dtype, opt, out, st, ws, c);
}

int lms_fit_host(const void *x, const void *y, int64_t n, int64_t h, int32_t dtype, const lms_options *opt,
                 lms_result *out, lms_stream_t stream)
{
    int rc = check_args(x, y, n, h, dtype, opt, out);
    if (rc) return rc;
    int dev;
    if (current_device(dev)) return LMS_ERR_CUDA;
    Choice c;
    rc = choose((int)n, (int)h, dtype, opt, dev, c);
    if (rc) return rc;
    const size_t esz = (dtype == LMS_F32) ? 4 : 2;
    const size_t in_bytes = ((size_t)n * esz + 255) / 256 * 256;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    rc = workspace(c.bytes + 2 * in_bytes, st, &ws);
    if (rc) return rc;
    unsigned char *base = static_cast<unsigned char *>(ws);
    unsigned char *dx = base + c.bytes;
    unsigned char *dy = dx + in_bytes;
    lms_result *dres = reinterpret_cast<lms_result *>(base + c.bytes - 256);
    if (cudaMemcpyAsync(dx, x, (size_t)n * esz, cudaMemcpyHostToDevice, st) != cudaSuccess) return LMS_ERR_CUDA;
    if (cudaMemcpyAsync(dy, y, (size_t)n * esz, cudaMemcpyHostToDevice, st) != cudaSuccess) return LMS_ERR_CUDA;
    rc = run_fit(dx, dy, (int)n, (int)h, dtype, opt, dres, st, ws, c);
    if (rc) return rc;
    if (cudaMemcpyAsync(out, dres, sizeof(lms_result), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LMS_ERR_CUDA;
    return LMS_OK;
}

int lms_fit_bnb(const void *x, const void *y, int64_t n, int64_t h, const float *seed_slope,
                const lms_options *opt, lms_result *out, lms_bnb_stats *stats, lms_stream_t stream)
{
    return fit_bnb_after(x, y, n, h, seed_slope, opt, out, stats, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

size_t lms_workspace_size(int64_t n, int32_t dtype, const lms_options *opt)
{
    int64_t h = 0;
    static const char dummy = 0;
    if (check_args(&dummy, &dummy, n, h, dtype, opt, &dummy)) return 0;
    int dev;
    if (current_device(dev)) return 0;
    Choice c;
    if (choose((int)n, (int)h, dtype, opt, dev, c)) return 0;
    const size_t esz = (dtype == LMS_F32) ? 4 : 2;
    return c.bytes + 2 * (((size_t)n * esz + 255) / 256 * 256);
}

int lms_set_workspace(void *device_buffer, size_t bytes)
{
    int dev;
    if (current_device(dev)) return LMS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    g_ws[dev].ext = device_buffer;
    g_ws[dev].ext_bytes = device_buffer ? bytes : 0;
    ++g_ws[dev].gen;
    return LMS_OK;
}

int lms_reserve(int64_t n, int32_t dtype, const lms_options *opt)
{
    const size_t b = lms_workspace_size(n, dtype, opt);
    if (!b) return LMS_ERR_ARG;
    void *ws;
    return workspace(b, nullptr, &ws);
}

const char *lms_status_str(int status)
{
    switch (status) {
        case LMS_OK: return "ok";
        case LMS_ERR_ARG: return "invalid argument";
        case LMS_ERR_RANGE: return "input out of range";
        case LMS_ERR_VERTICAL: return "all x equal (no pairwise slope)";
        case LMS_ERR_TIMEOUT: return "device wait timed out";
        case LMS_ERR_CUDA: return "CUDA runtime error";
        case LMS_ERR_WORKSPACE: return "workspace too small";
        case LMS_ERR_UNSUPPORTED: return "unsupported combination";
        case LMS_ERR_INTERNAL: return "device consistency check failed";
        case LMS_ERR_TOO_LARGE: return "n above the capacity of the no-allocation entry point";
        default: return "unknown status";
    }
}

const char *lms_version(void) { return "lms-gb300 0.1 (sm_103a)"; }

}  // extern "C"
