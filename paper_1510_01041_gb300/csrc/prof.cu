// prof.cu -- optional per-stage timing and launch counting.
//
// When enabled, every kernel launch of the library is bracketed by two CUDA
// events recorded on the stream it runs on; lms_profile_read() waits for
// them and returns the accumulated milliseconds per stage.  The launch
// counter always runs.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "lms.h"

namespace lms {
namespace {

struct Mark {
    int stage;
    cudaEvent_t a, b;
};

std::atomic<bool> g_on{false};
std::atomic<long long> g_launches{0};
std::atomic<long long> g_stage_launches[STAGE_COUNT];
std::mutex g_mu;
std::vector<Mark> g_marks;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

const char *const kNames[STAGE_COUNT] = {
    "pack", "sample", "sample_sort", "splitters", "count", "bucket_prefix", "bucket_scan", "scatter",
    "segsort", "segsort_big", "plan", "sweep_init", "sweep", "argmin", "plain", "other", "node_bounds", "seeds",
    "setnet", "hough", "tree"};

}  // namespace

bool profiling_on() { return g_on.load(std::memory_order_relaxed); }

void add_launches(long long count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

StageTimer::StageTimer(int stage, cudaStream_t st) : stage_(stage), st_(st), a_(nullptr)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    g_stage_launches[stage].fetch_add(1, std::memory_order_relaxed);
    if (g_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lock(g_mu);
        a_ = take_event();
        cudaEventRecord(a_, st_);
    }
}

StageTimer::~StageTimer()
{
    if (a_) {
        std::lock_guard<std::mutex> lock(g_mu);
        cudaEvent_t b = take_event();
        cudaEventRecord(b, st_);
        g_marks.push_back({stage_, a_, b});
    }
}

}  // namespace lms

using namespace lms;

extern "C" {

void lms_profile_enable(int on) { g_on.store(on != 0); }

int lms_profile_read(double *ms, int64_t *launches, int max_stages)
{
    std::lock_guard<std::mutex> lock(g_mu);
    const int ns = max_stages < STAGE_COUNT ? max_stages : STAGE_COUNT;
    for (int s = 0; s < ns; ++s) {
        if (ms) ms[s] = 0.0;
        if (launches) launches[s] = 0;
    }
    for (const Mark &m : g_marks) {
        cudaEventSynchronize(m.b);
        float t = 0.f;
        cudaEventElapsedTime(&t, m.a, m.b);
        if (m.stage < ns) {
            if (ms) ms[m.stage] += t;
            if (launches) launches[m.stage] += 1;
        }
        g_pool.push_back(m.a);
        g_pool.push_back(m.b);
    }
    g_marks.clear();
    return STAGE_COUNT;
}

const char *lms_stage_name(int stage)
{
    return (stage >= 0 && stage < STAGE_COUNT) ? kNames[stage] : "?";
}

int64_t lms_launch_count(void) { return g_launches.load(); }

}  // extern "C"
