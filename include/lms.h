/*
 * lms.h -- C ABI of the GB300 exact 2D Least Median of Squares line estimator.
 *
 * Problem (Shapira & Hassner, Sec. 1 Eq. 1 and Sec. 3.1): for points
 * (x_k, y_k), k = 0..n-1, and an order statistic h (default floor(n/2)+1),
 * find the line y = theta1 x + theta2 minimising the h-th smallest squared
 * residual.  Equivalently (Sec. 3.1) find the narrowest vertical slab holding
 * h points; the line bisects it and med_sq = (slab height / 2)^2.  By the
 * equioscillation property (Sec. 3.3) the optimal slope is one of the
 * pairwise slopes (y_j - y_i)/(x_j - x_i); the library examines every one of
 * them exactly (Algorithm 1, Sec. 3.4).
 *
 * Ties are broken by the lexicographic order of (slab height, theta1,
 * theta2) as exact rationals; (i, j) is then the smallest index pair whose
 * slope is theta1.  For int16 inputs every field of lms_result is exact and
 * reproducible bit for bit: theta1, theta2 and med_sq are each one IEEE
 * double operation on the exact integers.
 *
 * Conventions for every call:
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory of the current device; "host" pointers are ordinary host memory.
 *   - The caller owns all input and output buffers.  The library owns an
 *     internal per-device workspace (grown with cudaMalloc on demand) unless
 *     the caller installs one with lms_set_workspace.  lms_fit,
 *     lms_fit_host, lms_fit_bnb and lms_fit_learned on one device all use
 *     that one workspace: fits whose GPU work may overlap (different streams
 *     or host threads) race and must be ordered by the caller; many fits at
 *     once go through one lms_fit_batched call instead.  The workspace
 *     bookkeeping itself is locked, so the calls may come from any thread.
 *   - Device-pointer calls are asynchronous on `stream` (NULL = the legacy
 *     default stream); host-pointer calls synchronise before returning.
 *   - The return value reports argument and launch errors detected on the
 *     host.  The per-fit outcome is lms_result.status, written on the device.
 *   - No C++ exception crosses this interface.
 */
#ifndef LMS_H
#define LMS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LMS_API __attribute__((visibility("default")))
#else
#define LMS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st *lms_stream_t;

enum lms_status {
    LMS_OK = 0,
    LMS_ERR_ARG = 1,          /* n < 2, n > 65536, h outside [1, n], null pointer, bad enum */
    LMS_ERR_RANGE = 2,        /* float input that is not finite */
    LMS_ERR_VERTICAL = 3,     /* all x equal: no pairwise slope; result is the window at slope 0 */
    LMS_ERR_TIMEOUT = 4,      /* a bounded device wait expired */
    LMS_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    LMS_ERR_WORKSPACE = 6,    /* installed workspace too small (or growth needed during capture) */
    LMS_ERR_UNSUPPORTED = 7,  /* combination not implemented (e.g. plain algorithm with n > 1024) */
    LMS_ERR_INTERNAL = 8,     /* a device-side consistency check failed (reported, never silent) */
    LMS_ERR_TOO_LARGE = 9     /* n above the fixed capacity of lms_fit_noalloc */
};

enum lms_dtype {
    LMS_I16 = 0,              /* int16 coordinates, exact integer arithmetic */
    LMS_F32 = 1               /* float32 coordinates */
};

enum lms_algo {
    LMS_ALGO_AUTO = 0,        /* library choice */
    LMS_ALGO_PLAIN = 1,       /* sort the projections at every pairwise slope (n <= 1024) */
    LMS_ALGO_SWEEP = 2,       /* exact kinetic sweep over slope-sorted events */
    LMS_ALGO_BNB = 3,         /* seeded branch-and-bound over slope intervals + sweep of survivors */
    LMS_ALGO_PAPER = 4        /* the paper's own kernel layout (Sec. 3.6): 8x8-thread vertex blocks,
                                 one thread block and a shared-memory bitonic sort per vertex,
                                 then the reduction; int16, n <= 1024; an ablation of Table 1 */
};

typedef struct {
    int32_t algorithm;        /* enum lms_algo */
    int32_t sweepers;         /* kinetic-sweep workers per launch, 0 = auto */
    int32_t buckets;          /* slope buckets for event generation, 0 = auto */
    int32_t seed_mode;        /* branch-and-bound without a predicted slope: 0 = upper bound at
                                 quantiles of sampled pairwise slopes, 1 = at evenly spaced
                                 slope angles (no look at the data) */
    int32_t reserved[4];      /* must be zero */
} lms_options;

/* Result of one fit: 88 bytes, same layout on host and device. */
typedef struct {
    int64_t w_num, w_den;     /* slab height w = w_num / w_den, w_den = s_den */
    int64_t s_num, s_den;     /* theta1 = s_num / s_den, reduced, s_den > 0 */
    int64_t t_num, t_den;     /* theta2 = t_num / t_den, t_den = 2 s_den */
    double theta1, theta2;    /* the line y = theta1 x + theta2 */
    double med_sq;            /* (w/2)^2: the h-th smallest squared residual */
    int32_t i, j;             /* smallest pair (i < j) with slope theta1; -1 if none */
    int32_t status;           /* enum lms_status for this fit */
    int32_t algorithm;        /* enum lms_algo that produced it */
} lms_result;

/*
 * lms_fit -- exact LMS of one point set (Algorithm 1, Sec. 3.4).
 *   x, y    device arrays of n coordinates (int16_t or float, per dtype), SoA.
 *   n       2 <= n <= 65536 for int16 points (above 58112 points each
 *           sweeping warp keeps its position array in global memory);
 *           float points up to 32768 (larger: LMS_ERR_UNSUPPORTED).
 *   h       order statistic in [1, n]; 0 selects floor(n/2) + 1.
 *   dtype   enum lms_dtype.
 *   opt     NULL for defaults.
 *   out     device pointer to one lms_result.
 * Asynchronous on `stream`.  Returns LMS_OK or a host-detected error.
 */
LMS_API int lms_fit(const void *x, const void *y, int64_t n, int64_t h, int32_t dtype,
            const lms_options *opt, lms_result *out, lms_stream_t stream);

/*
 * lms_fit_host -- same as lms_fit with host arrays and a host result: copies
 * the coordinates to the device, fits, copies the result back and waits.
 * Returns LMS_OK or the error; out->status holds the fit's status.
 */
LMS_API int lms_fit_host(const void *x, const void *y, int64_t n, int64_t h, int32_t dtype,
                 const lms_options *opt, lms_result *out, lms_stream_t stream);

/* Branch-and-bound statistics (lms_fit_bnb). */
typedef struct {
    int64_t events_total;     /* pairs with distinct x: the candidate slopes */
    int64_t events_swept;     /* pairs in slope buckets that survived the bounds */
    int64_t nodes_evaluated;  /* slope intervals whose lower bound was computed */
    int64_t nodes_pruned;     /* intervals dropped (lower bound > upper bound) */
    int32_t buckets_total, buckets_swept;
    int32_t levels;           /* bisection levels */
    int32_t seeded;           /* 1 if a predicted slope chose the upper-bound slopes */
    double upper_bound;       /* slab height bound used for pruning, -1 if none */
} lms_bnb_stats;

/*
 * lms_fit_bnb -- exact LMS by branch-and-bound over slope intervals: an
 * upper bound from the exact window width at a few rounds of slopes (each
 * round zooming in on the narrowest window found so far), a lower bound for
 * every slope interval from the hulls of the projections over the interval,
 * intervals with lower bound > upper bound dropped, and the surviving
 * intervals swept exactly.  The result equals lms_fit's bit for bit (ties
 * are never pruned).
 *   seed_slope  device pointer to one float: a predicted slope; half of the
 *               first round's slopes are sampled slopes near it.  NULL: the
 *               first round takes evenly spaced quantiles of the sampled
 *               slopes (seed_mode 0) or evenly spaced angles (seed_mode 1).
 *   stats       host pointer (may be NULL).
 * Other arguments as lms_fit (int16 points, n <= 65536).  Every step,
 * including the interval tree, runs on the device: with stats == NULL the
 * call is asynchronous on `stream`; with stats it waits for the fit and
 * fills them (the first such call on a host thread allocates 256 bytes of
 * page-locked host memory, kept for that thread until the process exits).
 */
LMS_API int lms_fit_bnb(const void *x, const void *y, int64_t n, int64_t h, const float *seed_slope,
                        const lms_options *opt, lms_result *out, lms_bnb_stats *stats, lms_stream_t stream);

/*
 * Learned slope proposal: a set network (per point 2 -> 64 -> 64 ReLU, max
 * over the points, 64 -> 32 ReLU -> 2) that predicts the LMS line's slope
 * angle and intercept in a normalised frame; BF16 weights, FP32
 * accumulation, trained by its own forward/backward/Adam kernels.  Its
 * prediction only chooses where branch-and-bound takes its upper bound; the
 * answer stays exact.  Not in the paper (an extension of its method).
 *
 * Sets are given in CSR form: device int16 x[], y[] and device int64
 * offsets[B + 1].  pred (device, B x 4 floats): angle, normalised intercept,
 * slope, intercept.  targets (device, B x 2): angle and normalised intercept;
 * the frame of a set is its bounding box: centre (cx, cy), scale = half the
 * larger side, normalised intercept b = (theta2 - cy + theta1 * cx) / scale.
 * Loss = mean over sets of (angle error)^2 + intercept_weight (b error)^2.
 */
typedef struct lms_setnet lms_setnet;
LMS_API int lms_setnet_create(uint64_t seed, lms_setnet **net);   /* on the current device */
LMS_API void lms_setnet_destroy(lms_setnet *net);
LMS_API int64_t lms_setnet_param_count(void);
/* copy the FP32 master weights to (set = 0) or from (set = 1) a host array */
LMS_API int lms_setnet_params(lms_setnet *net, float *host, int64_t count, int32_t set);
LMS_API int lms_setnet_forward(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets,
                               int64_t B, float *pred, lms_stream_t stream);
/* loss gradient of the current weights (grads: device, param_count floats; loss: device float) */
LMS_API int lms_setnet_backward(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets,
                                int64_t B, const float *targets, float intercept_weight, float *grads,
                                float *loss, lms_stream_t stream);
/* one Adam step (beta 0.9 / 0.999) on the loss of the batch */
LMS_API int lms_setnet_train_step(lms_setnet *net, const int16_t *x, const int16_t *y, const int64_t *offsets,
                                  int64_t B, const float *targets, float intercept_weight, float lr,
                                  float *loss, lms_stream_t stream);
/* checkpoint: weights and optimiser state (synchronous) */
LMS_API int lms_setnet_save(const lms_setnet *net, const char *path);
LMS_API int lms_setnet_load(lms_setnet *net, const char *path);
/* the network predicts the slope of one set, branch-and-bound takes it as its
 * seed.  LMS_ERR_ARG (a null net, or any argument lms_fit_bnb refuses) is
 * returned before any work is queued. */
LMS_API int lms_fit_learned(lms_setnet *net, const void *x, const void *y, int64_t n, int64_t h,
                            const lms_options *opt, lms_result *out, lms_bnb_stats *stats,
                            lms_stream_t stream);
/* lms_fit_learned with host arrays x, y (int16, n <= 65536; page-locked
 * memory makes the copies asynchronous) and a host result: copies the points
 * into device staging owned by `net` (allocated on the first such call, kept
 * until lms_setnet_destroy), fits, copies the result back and waits for
 * `stream`.  One net must not run two host-buffer fits at once.  Without
 * statistics (stats NULL) and with profiling off, the device part of
 * repeated calls with the same n, h and options runs as one CUDA graph:
 * captured on a stream owned by `net` by the second such call and replayed
 * on `stream` by the later ones (the same kernels, without a host launch
 * call for each).  It is captured again after the workspace moves (it grows,
 * or lms_set_workspace installs another) or the net's per-set buffers grow,
 * and is freed by lms_setnet_destroy; a failed capture falls back to direct
 * calls for that key. */
LMS_API int lms_fit_learned_host(lms_setnet *net, const void *x, const void *y, int64_t n, int64_t h,
                                 const lms_options *opt, lms_result *out, lms_bnb_stats *stats,
                                 lms_stream_t stream);

/*
 * Batched fits of many point sets of uneven size (not in the paper: its
 * Hough application runs one LMS per accumulator peak; this runs them all).
 * lms_batch_plan_create sizes everything from the host offsets once: sets
 * with at most plain_max_n points (0 = 256, at most 256) go to one
 * persistent plain kernel over (set, run of slopes) work items in three
 * size classes; larger sets (up to 32768 points) each get the exact sweep
 * of every slope or, from 512 points on, the exact branch-and-bound, spread
 * over `streams` internal streams (0 = 8).  It allocates the plan's
 * device memory and waits for the device.
 *   offsets_host  B + 1 offsets of the sets in the x/y arrays (host).
 *   h_host        per-set order statistic (NULL: floor(n/2) + 1 each).
 * lms_fit_batched enqueues one batch on `stream` (forking to the plan's
 * streams and joining back with events): it allocates nothing and does not
 * synchronise, so it can be captured into a CUDA graph.  x, y: device int16
 * arrays; offsets_dev: device copy of the offsets; out: B device records.
 * One plan must not run two batches concurrently (they share its memory).
 */
typedef struct lms_batch_plan lms_batch_plan;
LMS_API int lms_batch_plan_create(const int64_t *offsets_host, int64_t B, const int32_t *h_host,
                                  int32_t plain_max_n, int32_t streams, lms_batch_plan **plan);
/* The same with the size from which a set is fitted by the exact
 * branch-and-bound (lms_fit_bnb's method, asynchronous, without statistics)
 * instead of the sweep of every slope: bnb_min_n 0 = 512 points (the value
 * lms_batch_plan_create uses), > 0 = that size (at least 257), < 0 = never.
 * The branch-and-bound's result equals the sweep's bit for bit. */
LMS_API int lms_batch_plan_create_ex(const int64_t *offsets_host, int64_t B, const int32_t *h_host,
                                     int32_t plain_max_n, int32_t streams, int32_t bnb_min_n,
                                     lms_batch_plan **plan);
LMS_API int lms_batch_plan_destroy(lms_batch_plan *plan);
LMS_API size_t lms_batch_plan_bytes(const lms_batch_plan *plan);
LMS_API int lms_fit_batched(lms_batch_plan *plan, const void *x, const void *y, const int64_t *offsets_dev,
                            lms_result *out, lms_stream_t stream);

/*
 * Line detection: standard Hough transform + exact LMS of every peak's
 * supporting points (Sec. 5).  For each of B binary images (device, uint8,
 * B x H x W, nonzero = edge pixel) with image-centre coordinates
 * (x - W/2, y - H/2): every edge pixel votes for theta_t = pi t / n_theta,
 * t < n_theta, in rho bin floor(x cos_t + y sin_t + n_rho/2) (clamped to
 * [0, n_rho); products and the sum each rounded to float, no fused
 * multiply-add); the top_k peaks per image are taken greedily in the order
 * (votes desc, t asc, rho asc), skipping bins within +-nms_theta and
 * +-nms_rho of a taken peak; the points within band_px of each peak's line
 * (rho at the bin centre) are fitted by exact LMS, with x and y swapped for
 * near-vertical peaks (|sin| < |cos|).
 *   max_points   0: fit every band point.  Otherwise a band holding more
 *             than max_points points is randomly subsampled before the fit
 *             (Sec. 5: the supporting points may be sampled to save time):
 *             point u of set k (k = image * top_k + peak, u its raster rank
 *             in the band) is kept iff the upper 32 bits of SplitMix64's
 *             output function applied to sample_seed ^ ((k << 32 | u) *
 *             0x9E3779B97F4A7C15) are below floor(2^32 max_points / count):
 *             about max_points points, reproducible from the seed.  The fit
 *             is the exact LMS of the kept points.
 *   cos_sin   optional device table of n_theta (cos, sin) float pairs; NULL:
 *             computed on the host as cos/sin in double rounded to float.
 *   acc_out   optional device int32 [B][n_theta][n_rho] receiving the votes.
 *   out       host array of B * top_k lms_line (peaks in greedy order).
 * Besides the LMS fit, each line carries the ordinary least-squares line of
 * the same fitted points (exact integer sums, one double division), for
 * comparisons such as the paper's Sec. 5 experiments.
 * Synchronous; allocates its scratch.
 */
typedef struct {
    int32_t theta_index, rho_index, votes;   /* the peak; theta_index = -1 if the image had fewer peaks */
    int32_t transposed;                      /* 1: x and y swapped before the fit */
    int32_t npoints;                         /* points within the band */
    int32_t nfit;                            /* points fitted (npoints unless subsampled) */
    int32_t pad[2];
    lms_result fit;                          /* status LMS_ERR_ARG if fewer than 2 points */
    double ols_theta1, ols_theta2;           /* least squares y = theta1 x + theta2 of the fitted points
                                                (fit frame); NaN when undefined (all x equal, < 2 points) */
} lms_line;
LMS_API int lms_hough_refine(const uint8_t *edges, int64_t B, int32_t H, int32_t W, int32_t n_theta,
                             int32_t n_rho, int32_t top_k, float band_px, int32_t nms_theta, int32_t nms_rho,
                             int32_t max_points, uint64_t sample_seed, const float *cos_sin, int32_t *acc_out,
                             lms_line *out, lms_stream_t stream);

/*
 * lms_workspace_size -- device bytes one lms_fit of this size needs.
 * lms_set_workspace  -- install a caller-owned device buffer (NULL restores
 *                       the internal one).  The buffer must stay valid and
 *                       unused by others while fits run on it.
 * lms_reserve        -- grow the internal workspace up front (e.g. before
 *                       capturing fits into a CUDA graph).
 */
LMS_API size_t lms_workspace_size(int64_t n, int32_t dtype, const lms_options *opt);
LMS_API int lms_set_workspace(void *device_buffer, size_t bytes);
LMS_API int lms_reserve(int64_t n, int32_t dtype, const lms_options *opt);

/*
 * Profiling (off by default).  lms_profile_enable(1) brackets every kernel
 * launch of the library with CUDA events on the launch's stream.
 * lms_profile_read waits for the recorded events, writes the accumulated
 * milliseconds and launch counts per stage (up to max_stages entries, either
 * pointer may be NULL), clears the record and returns the number of stages.
 * lms_stage_name names a stage; lms_launch_count counts every kernel this
 * library has launched since it was loaded.
 */
LMS_API void lms_profile_enable(int on);
LMS_API int lms_profile_read(double *ms, int64_t *launches, int max_stages);
LMS_API const char *lms_stage_name(int stage);
LMS_API int64_t lms_launch_count(void);

/*
 * lms_measure_int_peak -- measured int32 instruction throughput of the
 * current GPU (instructions per second over all SMs), the denominator of the
 * integer roofline reported for the LMS kernels.  A full-occupancy grid runs
 * eight independent dependency chains per thread for `iters` x 8 steps:
 *   kind 0  alternating add and xor (one add-class and one logic-class
 *           instruction per step),
 *   kind 1  32-bit multiply-add (one instruction per step).
 * Timed with CUDA events on `stream` (one warm-up launch first); synchronous.
 * Allocates and frees 64 bytes of device memory.  LMS_ERR_ARG for a bad kind,
 * iters outside [1, 2^24] or a null pointer.
 */
LMS_API int lms_measure_int_peak(int32_t kind, int64_t iters, double *ops_per_s, lms_stream_t stream);

/*
 * lms_fit_noalloc -- the plain fit (every pairwise slope, sort, window scan)
 * for callers that cannot have the library allocate device memory.  The
 * paper has no counterpart; it is an interface convenience.
 *
 * Who needs it: real-time or embedded loops that forbid allocation once
 * running (cudaMalloc and cudaFree can block and synchronise the device),
 * and frameworks that hand out all device memory from their own pools and
 * budgets.  lms_fit may grow an internal workspace with cudaMalloc; this
 * call never allocates or frees.
 *
 *   x, y    device arrays of n int16 coordinates.
 *   n       2 <= n <= LMS_NOALLOC_MAX_N; larger n returns LMS_ERR_TOO_LARGE.
 *   h       order statistic in [1, n]; 0 selects floor(n/2) + 1.
 *   out     device pointer to one lms_result (same result as lms_fit with
 *           LMS_ALGO_PLAIN, bit for bit).
 * Asynchronous on `stream`.
 *
 * Its only scratch is a fixed array of LMS_NOALLOC_MAX_WARPS * 32 bytes
 * (256 KiB) compiled into the library, present on every GPU that loads the
 * library until the process exits.  All calls share that array: calls whose
 * GPU work overlaps (other streams, other host threads) race and must not be
 * issued.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.
 */
#define LMS_NOALLOC_MAX_N 1024
#define LMS_NOALLOC_MAX_WARPS 8192
LMS_API int lms_fit_noalloc(const void *x, const void *y, int64_t n, int64_t h, lms_result *out,
                            lms_stream_t stream);

/* Human-readable name of a status code (static string). */
LMS_API const char *lms_status_str(int status);

/* Library version string. */
LMS_API const char *lms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LMS_H */
