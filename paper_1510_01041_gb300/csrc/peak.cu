// peak.cu -- measured int32 throughput of this GPU, the denominator of the
// integer roofline the benchmark reports for the LMS kernels (which are
// integer-ALU, shared-memory and latency work, not contractions).
//
// Every thread of a full-occupancy grid runs eight independent dependency
// chains; each step of a chain is one int32 instruction whose result the next
// step needs, so the compiler can neither drop nor merge the steps, and eight
// chains per thread at 64 warps per SM give the schedulers enough
// independent instructions to keep the integer pipes full.
//   kind 0: add/xor alternating (IADD-class and LOP-class instructions, the
//           bulk of the sweep's index arithmetic and comparisons)
//   kind 1: 32-bit multiply-add (a * b + c)
// The rate is instructions per second over the whole GPU, timed with CUDA
// events around one launch after a warm-up launch.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) k_int_peak(int iters, unsigned seed, unsigned *__restrict__ sink)
{
    unsigned a[PEAK_CHAINS];
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = t * (2u * c + 3u) + seed;
    const unsigned k1 = seed | 1u, k2 = seed * 0x9E3779B9u + 7u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) {
                if (KIND == 0) {
                    // two dependent instructions: add, then xor
                    a[c] = (a[c] + k1) ^ k2;
                } else {
                    // one multiply-add
                    a[c] = a[c] * k1 + k2;
                }
            }
        }
    }
    unsigned r = 0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) r ^= a[c];
    if (r == 0x12345678u) sink[0] = r;   // keeps the chains live; practically never taken
}

}  // namespace
}  // namespace lms

using namespace lms;

extern "C" int lms_measure_int_peak(int32_t kind, int64_t iters, double *ops_per_s, lms_stream_t stream)
{
    if (!ops_per_s || (kind != 0 && kind != 1) || iters < 1 || iters > (1LL << 24)) return LMS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return LMS_ERR_CUDA;
    }
    int per_sm = 0;
    const cudaError_t oe = kind == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int_peak<0>, PEAK_THREADS, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int_peak<1>, PEAK_THREADS, 0);
    if (oe != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return LMS_ERR_CUDA;
    }
    const int blocks = sms * per_sm;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = LMS_ERR_CUDA;
    float ms = 0.f;
    if (cudaMalloc(&sink, 64) != cudaSuccess) goto done;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up clocks and caches
        if (cudaEventRecord(a, st) != cudaSuccess) goto done;
        {
            StageTimer _t(STAGE_OTHER, st);
            if (kind == 0) k_int_peak<0><<<blocks, PEAK_THREADS, 0, st>>>((int)iters, 0x2545F491u, sink);
            else k_int_peak<1><<<blocks, PEAK_THREADS, 0, st>>>((int)iters, 0x2545F491u, sink);
        }
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess) goto done;
    }
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
        goto done;
    {
        const double per_step = kind == 0 ? 2.0 : 1.0;   // instructions per chain step
        const double ops = (double)blocks * PEAK_THREADS * (double)iters * 8.0 * PEAK_CHAINS * per_step;
        *ops_per_s = ops / (ms * 1e-3);
    }
    rc = LMS_OK;
done:
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    return rc;
}
