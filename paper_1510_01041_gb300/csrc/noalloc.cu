// noalloc.cu -- lms_fit_noalloc: the plain per-slope fit without any device
// allocation.
//
// Some callers cannot let a library allocate GPU memory: real-time or
// embedded loops that forbid allocation after start-up (cudaMalloc and
// cudaFree can block and synchronise the device), and frameworks that own
// all device memory through their own pools and budgets.  For them this
// entry point keeps its only scratch buffer -- the per-warp best windows
// that the final reduction reads -- in a fixed array compiled into the
// library.  The array lives on every GPU that loads the
// library until the process exits.
//
// Limits: int16 points, 2 <= n <= 1024 (the plain kernel's register sort),
// at most LMS_NOALLOC_MAX_WARPS warps of scratch (256 KiB).  All calls share
// the one array, so two calls whose work overlaps on the GPU (different
// streams, or different host threads) race and must not be issued.
//
// The device address of the array is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; make
// that first call before starting any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr int kNoallocMaxWarps = LMS_NOALLOC_MAX_WARPS;
constexpr int kMaxDevices = 64;

// Every warp of the plain kernel writes its own slot, so nothing in the array
// has to start at zero; stale slots of earlier calls are never read because
// the reduction only reads the slots of the warps this call launched.
static __device__ __align__(256) Cand g_noalloc_scratch[kNoallocMaxWarps];

std::mutex g_na_mu;
Cand *g_na_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (set up once),
// and that device's index.
int noalloc_scratch(Cand **out, int *device)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LMS_ERR_CUDA;
    *device = dev;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return LMS_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<Cand *>(p);
    }
    *out = g_na_ptr[dev];
    return LMS_OK;
}

}  // namespace
}  // namespace lms

using namespace lms;

extern "C" int lms_fit_noalloc(const void *x, const void *y, int64_t n, int64_t h, lms_result *out,
                               lms_stream_t stream)
{
    if (!x || !y || !out) return LMS_ERR_ARG;
    if (n < 2) return LMS_ERR_ARG;
    if (h == 0) h = n / 2 + 1;
    if (h < 1 || h > n) return LMS_ERR_ARG;
    if (n > LMS_NOALLOC_MAX_N) return LMS_ERR_TOO_LARGE;
    Cand *scratch = nullptr;
    int dev = 0, sms = 1;
    const int rc = noalloc_scratch(&scratch, &dev);
    if (rc) return rc;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LMS_ERR_CUDA;
    }
    // warps: up to 32 per SM, at least ~4 slopes each, a multiple of 8, and
    // never more than the array holds
    const long long npairs = n * (n - 1) / 2;
    long long warps = (long long)(sms > 0 ? sms : 1) * 32;
    if ((npairs + 3) / 4 < warps) warps = (npairs + 3) / 4;
    warps = (warps + 7) / 8 * 8;
    if (warps < 8) warps = 8;
    if (warps > kNoallocMaxWarps) warps = kNoallocMaxWarps / 8 * 8;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (launch_plain((const short *)x, (const short *)y, (int)n, (int)h, scratch, (int)warps, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    if (launch_argmin(scratch, (int)warps, out, LMS_ALGO_PLAIN, nullptr, st) != cudaSuccess)
        return LMS_ERR_CUDA;
    return LMS_OK;
}
