// kernels.cuh -- host-side launch declarations for the LMS kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lms {

// Stages of a fit, for per-launch timing (prof.cu).
enum Stage {
    STAGE_PACK, STAGE_SAMPLE, STAGE_SAMPLE_SORT, STAGE_SPLITTERS, STAGE_COUNT_PAIRS, STAGE_PREFIX,
    STAGE_SCAN, STAGE_SCATTER, STAGE_SEGSORT, STAGE_SEGSORT_BIG, STAGE_PLAN, STAGE_INIT, STAGE_SWEEP,
    STAGE_ARGMIN, STAGE_PLAIN, STAGE_OTHER, STAGE_NODE_LB, STAGE_SEEDS, STAGE_SETNET, STAGE_HOUGH, STAGE_TREE,
    STAGE_COUNT
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

// Slope-key policies for the event pipeline: key() returns false when the
// pair has no slope (equal x) and otherwise an int64 key that orders slopes.
struct KeyI16 {   // packed int16 points: exact key floor(dy 2^32 / dx)
    static __device__ __forceinline__ bool key(const void *pts, int i, int j, long long &k)
    {
        const int *xy = static_cast<const int *>(pts);
        int dy, dx;
        if (!pair_slope(__ldg(&xy[i]), __ldg(&xy[j]), dy, dx)) return false;
        k = slope_key(dy, dx);
        return true;
    }
    // float slope dy * (1 / dx), relative error below 2^-22; false when x_i == x_j
    static __device__ __forceinline__ bool approx(const void *pts, int i, int j, float &sl)
    {
        const int *xy = static_cast<const int *>(pts);
        int dy, dx;
        if (!pair_slope(__ldg(&xy[i]), __ldg(&xy[j]), dy, dx)) return false;
        sl = __fmul_rn((float)dy, __frcp_rn((float)dx));
        return true;
    }
};
struct KeyF32 {   // float2 points: the double slope dy/dx as order-preserving bits
    static __device__ __forceinline__ bool key(const void *pts, int i, int j, long long &k)
    {
        const float2 *P = static_cast<const float2 *>(pts);
        const float2 a = P[i], b = P[j];
        double dx = (double)b.x - (double)a.x, dy = (double)b.y - (double)a.y;
        if (dx == 0.0) return false;
        if (dx < 0.0) { dx = -dx; dy = -dy; }
        const double sl = __ddiv_rn(dy, dx);
        const long long bits = sl == 0.0 ? 0LL : __double_as_longlong(sl);
        k = bits < 0 ? (bits ^ 0x7fffffffffffffffLL) : bits;
        return true;
    }
    static __device__ __forceinline__ bool approx(const void *pts, int i, int j, float &sl)
    {
        const float2 *P = static_cast<const float2 *>(pts);
        const double dx = (double)P[j].x - (double)P[i].x, dy = (double)P[j].y - (double)P[i].y;
        if (dx == 0.0) return false;
        sl = (float)(dy / dx);
        return true;
    }
};

// ---------------------------------------------------------------- plain path
int plain_elems(int n);
cudaError_t launch_plain(const short *x, const short *y, int n, int h, Cand *cands, int nwarps_total,
                         cudaStream_t st);

// ---------------------------------------------------------------- the paper's kernel layout
size_t paper_bytes(int n);
// vertices, then one block per vertex; *cands / *count: the records for the argmin
cudaError_t launch_paper(const short *x, const short *y, int n, int h, void *ws, Cand **cands, long long *count,
                         cudaStream_t st);

// ---------------------------------------------------------------- sweep path
constexpr int SEG_CAP = 16384;   // events a bucket may hold to be sorted in shared memory
constexpr int SEG_REPAIR_MAX = 64;   // odd-even passes a bucket sort may spend on cells of equal shifted keys
constexpr int BND_MAX = 16384;   // slope-bucket boundaries (power of two, shared memory)
constexpr int SORT_SMEM_N = 8192;  // sweep start orders sorted in shared memory up to this n

// Device scratch of one sweep-path fit; carved out of the workspace by the host.
struct SweepPlan {
    int n, h;
    int S;             // sampled pairs (power of two, >= 1024)
    int B;             // target number of quantile buckets
    int C;             // CTAs of the count / scatter passes
    int W;             // slope ranges (each starts with a sort of the points)
    int G;             // sweeping warps of the persistent sweep kernel (G < W + spb)
    int spb;           // sweeping warps per sweep CTA
    bool xy_smem;      // sweep CTAs keep all points in shared memory
    bool pos_smem;     // sweeping warps keep the position array in shared memory (else gpos)
    long long emax;    // n (n - 1) / 2
    // device buffers
    int *xy;                   // [n] packed points
    long long *skeys;          // [S] sampled slope keys
    long long *skeys2;         // [S] merge ping-pong
    long long *bnd;            // [BND_MAX] bucket boundaries, padded with INT64_MAX
    int *meta;                 // [16] 0 nbnd, 1 P2, 2 oversize count, 3 error flags, 4 range counter,
                               //      5 pairs with distinct x, 6 listed kept pairs (restricted count),
                               //      7 / 8 events covered by the ranges / events there are,
                               //      10 valid sampled keys
    unsigned *hist;            // [C][BND_MAX] per-CTA bucket counts, then offsets
    unsigned *base;            // [BND_MAX + 1] bucket starts; base[NB] = E
    int *oversize;             // [BND_MAX] buckets too large for the shared-memory sort
    unsigned *ev;              // [emax] events
    unsigned *ev2;             // [emax] merge copy for buckets above SEG_CAP; before the bucket sorts,
                               //        the list of kept pairs of a restricted count
    unsigned *range;           // [2W] range event bounds
    unsigned short *orders;    // [W][n] start orders
    unsigned long long *gsort; // [W][2P] words, then [W][P] 16-bit payloads: start sorts when n > SORT_SMEM_N
    Cand *cands;               // [W + G] range-start + sweeping-warp candidates
    unsigned short *gpos;      // [G][n] positions of the sweeping warps when !pos_smem (else null)
    // A restricted pass with resplit set sorts its kept events in buckets of
    // their own: splitters from a sample of the listed pairs (about
    // RESPLIT_PER events a bucket) instead of the buckets of all pairs, of
    // which the kept ones can be far above SEG_CAP.
    bool resplit;
    long long *bnd2;           // [BND_MAX] boundaries of the kept events' buckets
    unsigned *base2;           // [BND_MAX + 1] their starts
    int *meta2;                // [16] their nbnd, P2 and oversize count (layout of meta)
};
constexpr int RESPLIT_PER = 4096;    // kept events per bucket of a resplit pass
constexpr int RESPLIT_S = 32768;     // sampled listed pairs of a resplit pass (at most S)

size_t sweep_plan_bytes(const SweepPlan &p);
// concurrent: the fit shares the GPU with other fits (batch plans)
void sweep_plan_configure(SweepPlan &p, int n, int h, int sms, int want_w, int want_b, bool concurrent = false);
void sweep_plan_carve(SweepPlan &p, void *ws);
cudaError_t launch_sweep(const SweepPlan &p, const short *x, const short *y, cudaStream_t st);
// the two halves of launch_sweep: bucket counts and starts (prepare), then
// scatter of the kept buckets' events, bucket sorts and the sweep (finish)
cudaError_t launch_sweep_prepare(const SweepPlan &p, const short *x, const short *y, cudaStream_t st);
// plan = false: the caller has written the range bounds (any event offsets
// inside runs of kept buckets); they are moved to group starts on the device
cudaError_t launch_sweep_finish(const SweepPlan &p, const unsigned char *keep, cudaStream_t st, bool plan,
                                bool listed = false);
const long long *sorted_sample(const SweepPlan &p);
// generic halves of the event pipeline (sample .. bucket starts; scatter .. plan)
template <class G> cudaError_t launch_events_prepare(const SweepPlan &p, const void *pts, cudaStream_t st);
template <class G>
cudaError_t launch_events_finish(const SweepPlan &p, const void *pts, const unsigned char *keep, cudaStream_t st,
                                 bool plan, bool listed = false);
// A restricted pass (the branch-and-bound's) lists the pairs whose exact
// slope key lies in a kept bucket; the kept buckets form at most PRE_MAX
// covers, given as key ranges [cov[2c], cov[2c + 1]) (unused covers empty).
constexpr int PRE_MAX = 32;
// the sample half of the prepare step (pack, sample, sort, splitters), and
// the restricted count (the kept pairs listed into ev2 and counted per
// bucket, then prefix and scan)
cudaError_t launch_sweep_sample(const SweepPlan &p, const short *x, const short *y, cudaStream_t st);
// scratch: band_scratch_bytes(n); distinct_x: also count the pairs with
// distinct x into meta[5]
size_t band_scratch_bytes(int n);
cudaError_t launch_sweep_count(const SweepPlan &p, const unsigned char *keep, const long long *cov, void *scratch,
                               bool distinct_x, cudaStream_t st);
// per-bucket counts of the valid sampled pairs into counts[0 .. NB)
cudaError_t launch_sample_counts(const SweepPlan &p, unsigned *counts, cudaStream_t st);
// float32 points: event pipeline on the double slope key, double-precision
// sweep, reduction into `out` (device).  fscratch: sweep_f32_extra_bytes.
cudaError_t launch_sweep_f32_fit(const SweepPlan &p, const float *x, const float *y, void *fscratch,
                                 lms_result *out, cudaStream_t st);
size_t sweep_f32_extra_bytes(int n, int W);

// ---------------------------------------------------------------- branch and bound
size_t bnb_extra_bytes(int n, int sms);
// pred_ready: when not null, an event the step that reads pred_dev waits for
// (the prediction may be computed on another stream meanwhile).
int run_bnb(const SweepPlan &p, const short *x, const short *y, const float *pred_dev, int seed_mode, lms_result *out,
            lms_bnb_stats *stats, void *extra, int sms, cudaStream_t st, cudaEvent_t pred_ready = nullptr);
// lms_fit_bnb with the event above
int fit_bnb_after(const void *x, const void *y, int64_t n, int64_t h, const float *seed_slope, const lms_options *opt,
                  lms_result *out, lms_bnb_stats *stats, cudaStream_t st, cudaEvent_t pred_ready);
// the argument checks of lms_fit_bnb (LMS_OK or LMS_ERR_ARG), no device work
int check_bnb_args(const void *x, const void *y, int64_t n, int64_t h, const lms_options *opt, const void *out);
// changes whenever the current device's workspace buffer may have moved (a
// captured graph that uses it must then be captured again)
unsigned long long workspace_generation();
// whether per-launch profiling events are on; launches run by replaying a
// captured graph, added to the launch counter
bool profiling_on();
void add_launches(long long count);

// ---------------------------------------------------------------- argmin
cudaError_t launch_argmin(const Cand *cands, int count, lms_result *out, int algorithm, const int *err,
                          cudaStream_t st);

}  // namespace lms
