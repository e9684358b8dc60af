// kernels.cuh -- host-side launch declarations for the LMS kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lms {

// Stages of a fit, for per-launch timing (prof.cu).
enum Stage {
    STAGE_PACK, STAGE_SAMPLE, STAGE_SAMPLE_SORT, STAGE_SPLITTERS, STAGE_COUNT_PAIRS, STAGE_PREFIX,
    STAGE_SCAN, STAGE_SCATTER, STAGE_SEGSORT, STAGE_SEGSORT_BIG, STAGE_PLAN, STAGE_INIT, STAGE_SWEEP,
    STAGE_ARGMIN, STAGE_PLAIN, STAGE_OTHER, STAGE_COUNT
};

// Counts one kernel launch and, when profiling is on, brackets it with CUDA
// events on its stream.  Construct it right before the launch.
class StageTimer {
  public:
    StageTimer(int stage, cudaStream_t st);
    ~StageTimer();
    StageTimer(const StageTimer &) = delete;
    StageTimer &operator=(const StageTimer &) = delete;

  private:
    int stage_;
    cudaStream_t st_;
    cudaEvent_t a_;
};

// ---------------------------------------------------------------- plain path
int plain_elems(int n);
cudaError_t launch_plain(const short *x, const short *y, int n, int h, Cand *cands, int nwarps_total,
                         cudaStream_t st);

// ---------------------------------------------------------------- sweep path
constexpr int SEG_CAP = 16384;   // events a bucket may hold to be sorted in shared memory
constexpr int BND_MAX = 16384;   // slope-bucket boundaries (power of two, shared memory)
constexpr int SORT_SMEM_N = 8192;  // sweep start orders sorted in shared memory up to this n

// Device scratch of one sweep-path fit; carved out of the workspace by the host.
struct SweepPlan {
    int n, h;
    int S;             // sampled pairs (power of two, >= 1024)
    int B;             // target number of quantile buckets
    int C;             // CTAs of the count / scatter passes
    int W;             // sweepers
    int spb;           // sweepers (warps) per sweep CTA
    bool xy_smem;      // sweep CTAs keep all points in shared memory
    long long emax;    // n (n - 1) / 2
    // device buffers
    int *xy;                   // [n] packed points
    long long *skeys;          // [S] sampled slope keys
    long long *skeys2;         // [S] merge ping-pong
    long long *bnd;            // [BND_MAX] bucket boundaries, padded with INT64_MAX
    int *meta;                 // [8] 0 nbnd, 1 P2, 2 oversize count, 3 error flags
    unsigned *hist;            // [C][BND_MAX] per-CTA bucket counts, then offsets
    unsigned *base;            // [BND_MAX + 1] bucket starts; base[NB] = E
    int *oversize;             // [BND_MAX] buckets too large for the shared-memory sort
    unsigned *ev;              // [emax] events
    unsigned *range;           // [2W] sweeper event ranges
    unsigned short *orders;    // [W][n] start orders
    unsigned long long *gsort; // [W][P] global sort scratch when n > SORT_SMEM_N
    Cand *cands;               // [2W] init + sweep candidates
};

size_t sweep_plan_bytes(int n, int W, int C, int S);
void sweep_plan_configure(SweepPlan &p, int n, int h, int sms, int want_w, int want_b);
void sweep_plan_carve(SweepPlan &p, void *ws);
cudaError_t launch_sweep(const SweepPlan &p, const short *x, const short *y, cudaStream_t st);
// the two halves of launch_sweep: bucket counts and starts (prepare), then
// scatter of the kept buckets' events, bucket sorts and the sweep (finish)
cudaError_t launch_sweep_prepare(const SweepPlan &p, const short *x, const short *y, cudaStream_t st);
// plan = false: the caller has written the sweeper ranges itself
cudaError_t launch_sweep_finish(const SweepPlan &p, const unsigned char *keep, cudaStream_t st, bool plan);
const long long *sorted_sample(const SweepPlan &p);

// ---------------------------------------------------------------- branch and bound
size_t bnb_extra_bytes(int n, int sms);
int run_bnb(const SweepPlan &p, const short *x, const short *y, const float *pred_dev, int seed_mode, lms_result *out,
            lms_bnb_stats *stats, void *extra, int sms, cudaStream_t st);

// ---------------------------------------------------------------- argmin
cudaError_t launch_argmin(const Cand *cands, int count, lms_result *out, int algorithm, const int *err,
                          cudaStream_t st);

}  // namespace lms
