/*
 * lms_oracle.c -- CPU oracle for the exact 2D Least Median of Squares (LMS)
 * line estimator of Shapira & Hassner, "GPU-Based Computation of 2D Least
 * Median of Squares with Applications to Fast and Robust Line Detection".
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never links, loads or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Sec. 1 Eq. 1; Sec. 3.1 slab; Sec. 3.2 bracelet;
 * Sec. 3.3 equioscillation; Sec. 3.4 Algorithm 1 and its correctness note):
 *   For points (x_k, y_k) and an order statistic h (default floor(n/2)+1),
 *   LMS = min over lines of the h-th smallest squared residual.  For a fixed
 *   slope s the best intercept puts the line in the middle of the narrowest
 *   vertical window holding h of the projections z_k = y_k - s x_k, so the
 *   h-th smallest |residual| is w(s)/2 with w(s) that window's width (the
 *   slab height of Sec. 3.1).  Between two consecutive pairwise slopes the
 *   sorted order of z is fixed, each window width is linear in s and w(s) is
 *   a minimum of linear functions, hence concave; on the unbounded end
 *   pieces it is monotone toward the finite end.  So the minimum is attained
 *   at a pairwise slope (the vertices of the dual arrangement, Sec. 3.3).
 *   The oracle returns, over every pairwise slope s = dy/dx (dx != 0) and
 *   every window of h consecutive sorted projections at s, the
 *   lexicographic minimum of (w, theta1 = s, theta2 = window centre), all as
 *   exact rationals, and the smallest index pair (i < j) whose slope is
 *   theta1.  med_sq = (w/2)^2.
 *
 * Two independent implementations:
 *   O1 oracle_lms_*_brute: every pair's slope, a full sort of the
 *      projections, every window (Algorithm 1 read literally, with all
 *      windows rather than only upward bracelets).
 *   O2 oracle_lms_*_sweep: the vertical sweep of the dual arrangement cited
 *      in Sec. 2 (Souvaine & Steele): events sorted by an exact rational
 *      comparator, the order kept between events, every run of equal
 *      projections re-sorted at its event and only windows with an end in a
 *      re-sorted run re-scored; a full scan at the first event.
 *
 * Arithmetic: coordinates are int64 (int16 inputs widen; float32 inputs are
 * scaled by one power of two into exact integers), projections are
 * key_k = y_k * sd - x_k * sn = z_k * sd in __int128, and rationals are
 * compared through exact 256-bit cross products.  No floating point is used
 * until the final conversion of the exact result to doubles.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

enum {
    OR_OK = 0,
    OR_ERR_ARG = 1,
    OR_ERR_VERTICAL = 3,
    OR_ERR_UNSUPPORTED = 7,
    OR_ERR_NOMEM = 8
};

/* Result as handed back to Python.  Integer fields hold the exact rationals
 * when they fit in int64 (always for int16 inputs), else 0 with ints_valid=0. */
typedef struct {
    int64_t w_num, w_den;   /* slab height w = w_num / w_den (scaled by 2^-scale_exp) */
    int64_t s_num, s_den;   /* theta1 = s_num / s_den, reduced, s_den > 0 */
    int64_t t_num, t_den;   /* theta2 = t_num / t_den (scaled by 2^-scale_exp), t_den = 2 s_den */
    double theta1, theta2, med_sq;
    int32_t i, j;           /* smallest pair (i < j) with slope theta1; -1 if none */
    int32_t status;
    int32_t scale_exp;      /* float inputs: coordinates were multiplied by 2^scale_exp */
    int32_t ints_valid;
    int32_t pad;
} oracle_result;

typedef struct {
    i128 w, sn, sd, t;      /* width*sd, slope sn/sd, (sum of window end keys) */
    int64_t i, j;
    int valid;
} cand_t;

/* ------------------------------------------------------------------ exact */

static void mul_u128(u128 a, u128 b, u128 *hi, u128 *lo)
{
    uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1;
    u128 p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
    *lo = (mid << 64) | (uint64_t)p00;
    *hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

static int sgn128(i128 v) { return (v > 0) - (v < 0); }
static u128 abs128(i128 v) { return v < 0 ? (u128)(-v) : (u128)v; }

/* sign of a/b - c/d for b, d > 0 (sign of a*d - c*b), exact. */
static int cmp_frac(i128 a, i128 b, i128 c, i128 d)
{
    int sa = sgn128(a), sc = sgn128(c);
    if (sa != sc) return sa > sc ? 1 : -1;
    if (sa == 0) return 0;
    u128 h1, l1, h2, l2;
    mul_u128(abs128(a), (u128)d, &h1, &l1);
    mul_u128(abs128(c), (u128)b, &h2, &l2);
    int m = (h1 != h2) ? (h1 > h2 ? 1 : -1) : (l1 != l2 ? (l1 > l2 ? 1 : -1) : 0);
    return sa > 0 ? m : -m;
}

static u128 gcd_u128(u128 a, u128 b)
{
    while (b) { u128 r = a % b; a = b; b = r; }
    return a;
}

/* Reduced slope (sn/sd, sd > 0) of the pair (i, j); returns 0 if x_i == x_j. */
static int pair_slope(const int64_t *x, const int64_t *y, int64_t i, int64_t j,
                      i128 *sn, i128 *sd)
{
    i128 dx = (i128)x[j] - x[i], dy = (i128)y[j] - y[i];
    if (dx == 0) return 0;
    if (dx < 0) { dx = -dx; dy = -dy; }
    u128 g = gcd_u128(abs128(dy), (u128)dx);
    if (g == 0) g = 1;
    *sn = dy / (i128)g;
    *sd = dx / (i128)g;
    return 1;
}

/* Lexicographic order on (w, theta1, theta2, i, j). */
static int better(const cand_t *a, const cand_t *b)
{
    if (!a->valid) return 0;
    if (!b->valid) return 1;
    int c = cmp_frac(a->w, a->sd, b->w, b->sd);
    if (c) return c < 0;
    c = cmp_frac(a->sn, a->sd, b->sn, b->sd);
    if (c) return c < 0;
    c = cmp_frac(a->t, a->sd, b->t, b->sd);
    if (c) return c < 0;
    if (a->i != b->i) return a->i < b->i;
    return a->j < b->j;
}

static int cmp_i128(const void *pa, const void *pb)
{
    i128 a = *(const i128 *)pa, b = *(const i128 *)pb;
    return (a > b) - (a < b);
}

/* w(s) at slope sn/sd: full sort of all projections, narrowest window of h,
 * first (lowest) such window.  keys: scratch of n entries. */
static void eval_slope(const int64_t *x, const int64_t *y, int64_t n, int64_t h,
                       i128 sn, i128 sd, i128 *keys, cand_t *out)
{
    for (int64_t k = 0; k < n; ++k)
        keys[k] = (i128)y[k] * sd - (i128)x[k] * sn;
    qsort(keys, (size_t)n, sizeof(i128), cmp_i128);
    int64_t best_a = 0;
    i128 best_w = keys[h - 1] - keys[0];
    for (int64_t a = 1; a + h - 1 < n; ++a) {
        i128 w = keys[a + h - 1] - keys[a];
        if (w < best_w) { best_w = w; best_a = a; }
    }
    out->w = best_w;
    out->t = keys[best_a] + keys[best_a + h - 1];
    out->sn = sn;
    out->sd = sd;
    out->valid = 1;
}

/* ------------------------------------------------------------ conversion */

static int fits64(i128 v) { return v >= (i128)INT64_MIN && v <= (i128)INT64_MAX; }

static void finalize(const cand_t *c, int status, int scale_exp, oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    out->status = status;
    out->scale_exp = scale_exp;
    out->i = (int32_t)c->i;
    out->j = (int32_t)c->j;
    i128 wden = c->sd, tden = 2 * c->sd;
    out->ints_valid = fits64(c->w) && fits64(c->t) && fits64(c->sn) && fits64(tden);
    if (out->ints_valid) {
        out->w_num = (int64_t)c->w;  out->w_den = (int64_t)wden;
        out->s_num = (int64_t)c->sn; out->s_den = (int64_t)c->sd;
        out->t_num = (int64_t)c->t;  out->t_den = (int64_t)tden;
    }
    /* One IEEE operation per quantity on exact integers (int16 inputs). */
    out->theta1 = (double)c->sn / (double)c->sd;
    out->theta2 = ldexp((double)c->t / (double)tden, -scale_exp);
    double r = ldexp((double)c->w / (double)(2 * wden), -scale_exp);
    out->med_sq = r * r;
}

/* ------------------------------------------------------------------- O1 */

static int brute_core(const int64_t *x, const int64_t *y, int64_t n, int64_t h,
                      cand_t *best_out)
{
    cand_t best = {0};
    int failed = 0;
#pragma omp parallel
    {
        cand_t local = {0};
        i128 *keys = (i128 *)malloc(sizeof(i128) * (size_t)n);
        if (!keys) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < n; ++i) {
                for (int64_t j = i + 1; j < n; ++j) {
                    i128 sn, sd;
                    if (!pair_slope(x, y, i, j, &sn, &sd)) continue;
                    cand_t c;
                    eval_slope(x, y, n, h, sn, sd, keys, &c);
                    c.i = i; c.j = j;
                    if (better(&c, &local)) local = c;
                }
            }
            free(keys);
        }
#pragma omp critical
        {
            if (better(&local, &best)) best = local;
        }
    }
    if (failed) return OR_ERR_NOMEM;
    *best_out = best;
    return OR_OK;
}

/* ------------------------------------------------------------------- O2 */

typedef struct { uint16_t i, j; } ev_t;

typedef struct { const int64_t *x, *y; } coords_t;

static void ev_slope(const coords_t *c, const ev_t *e, i128 *dy, i128 *dx)
{
    i128 ddx = (i128)c->x[e->j] - c->x[e->i], ddy = (i128)c->y[e->j] - c->y[e->i];
    if (ddx < 0) { ddx = -ddx; ddy = -ddy; }
    *dy = ddy; *dx = ddx;
}

/* Events ordered by exact slope dy/dx, then by (i, j). */
static int ev_cmp(const void *pa, const void *pb, void *ctx)
{
    const ev_t *a = (const ev_t *)pa, *b = (const ev_t *)pb;
    i128 ay, ax, by, bx;
    ev_slope((const coords_t *)ctx, a, &ay, &ax);
    ev_slope((const coords_t *)ctx, b, &by, &bx);
    i128 l = ay * bx, r = by * ax;          /* |.| < 2^126 */
    if (l != r) return l < r ? -1 : 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    return (a->j > b->j) - (a->j < b->j);
}

static int same_slope(const coords_t *c, const ev_t *a, const ev_t *b)
{
    i128 ay, ax, by, bx;
    ev_slope(c, a, &ay, &ax);
    ev_slope(c, b, &by, &bx);
    return ay * bx == by * ax;
}

/* Chunked parallel sort: each thread sorts a chunk, then chunks merge pairwise. */
static int sort_events(ev_t *ev, size_t m, coords_t *ctx)
{
    int T = omp_get_max_threads();
    if (T < 1) T = 1;
    if (m < (size_t)1 << 16) T = 1;
    size_t *bnd = (size_t *)malloc(sizeof(size_t) * (size_t)(T + 1));
    if (!bnd) return OR_ERR_NOMEM;
    for (int t = 0; t <= T; ++t) bnd[t] = m * (size_t)t / (size_t)T;
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < T; ++t)
        qsort_r(ev + bnd[t], bnd[t + 1] - bnd[t], sizeof(ev_t), ev_cmp, ctx);
    if (T > 1) {
        ev_t *tmp = (ev_t *)malloc(sizeof(ev_t) * m);
        if (!tmp) { free(bnd); return OR_ERR_NOMEM; }
        ev_t *src = ev, *dst = tmp;
        for (int width = 1; width < T; width *= 2) {
#pragma omp parallel for schedule(dynamic, 1)
            for (int t = 0; t < T; t += 2 * width) {
                size_t a0 = bnd[t];
                size_t a1 = bnd[t + width < T ? t + width : T];
                size_t b1 = bnd[t + 2 * width < T ? t + 2 * width : T];
                size_t p = a0, q = a1, o = a0;
                while (p < a1 && q < b1)
                    dst[o++] = (ev_cmp(&src[q], &src[p], ctx) < 0) ? src[q++] : src[p++];
                while (p < a1) dst[o++] = src[p++];
                while (q < b1) dst[o++] = src[q++];
            }
            ev_t *s = src; src = dst; dst = s;
        }
        if (src != ev) memcpy(ev, src, sizeof(ev_t) * m);
        free(tmp);
    }
    free(bnd);
    return OR_OK;
}

typedef struct {
    const int64_t *x, *y;
    const i128 *key;
} order_ctx_t;

/* Just-before order at an event slope: by projection, then x ascending, then index. */
static int before_cmp(const void *pa, const void *pb, void *vctx)
{
    const order_ctx_t *c = (const order_ctx_t *)vctx;
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (c->key[a] != c->key[b]) return c->key[a] < c->key[b] ? -1 : 1;
    if (c->x[a] != c->x[b]) return c->x[a] < c->x[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* Just-after order inside a run of equal projections: x descending, then index. */
static int after_cmp(const void *pa, const void *pb, void *vctx)
{
    const order_ctx_t *c = (const order_ctx_t *)vctx;
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (c->x[a] != c->x[b]) return c->x[a] > c->x[b] ? -1 : 1;
    return (a > b) - (a < b);
}

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

static i128 proj(const int64_t *x, const int64_t *y, int32_t k, i128 sn, i128 sd)
{
    return (i128)y[k] * sd - (i128)x[k] * sn;
}

static void score_window(const int64_t *x, const int64_t *y, const int32_t *order,
                         int64_t h, int64_t a, i128 sn, i128 sd, int64_t pi, int64_t pj,
                         cand_t *best)
{
    cand_t c;
    i128 lo = proj(x, y, order[a], sn, sd), hi = proj(x, y, order[a + h - 1], sn, sd);
    c.w = hi - lo;
    c.t = lo + hi;
    c.sn = sn; c.sd = sd; c.i = pi; c.j = pj; c.valid = 1;
    if (better(&c, best)) *best = c;
}

static int sweep_core(const int64_t *x, const int64_t *y, int64_t n, int64_t h,
                      cand_t *best_out)
{
    if (n > 65536) return OR_ERR_UNSUPPORTED;
    /* all pairs with dx != 0 */
    size_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (x[i] != x[j]) ++m;
    if (m == 0) { best_out->valid = 0; return OR_OK; }
    ev_t *ev = (ev_t *)malloc(sizeof(ev_t) * m);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *plist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *flag = (char *)calloc((size_t)n, 1);
    i128 *key = (i128 *)malloc(sizeof(i128) * (size_t)n);
    if (!ev || !order || !pos || !plist || !tmp || !flag || !key) {
        free(ev); free(order); free(pos); free(plist); free(tmp); free(flag); free(key);
        return OR_ERR_NOMEM;
    }
    {
        size_t o = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j)
                if (x[i] != x[j]) { ev[o].i = (uint16_t)i; ev[o].j = (uint16_t)j; ++o; }
    }
    coords_t cc = { x, y };
    int rc = sort_events(ev, m, &cc);
    if (rc != OR_OK) goto done;

    cand_t best = {0};
    order_ctx_t oc = { x, y, key };
    size_t ga = 0;
    int first = 1;
    while (ga < m) {
        size_t gb = ga + 1;
        while (gb < m && same_slope(&cc, &ev[ga], &ev[gb])) ++gb;
        i128 sn, sd;
        pair_slope(x, y, ev[ga].i, ev[ga].j, &sn, &sd);
        /* events are sorted by (slope, i, j): the group's first is its smallest pair */
        int64_t pi = ev[ga].i, pj = ev[ga].j;
        if (first) {
            for (int64_t k = 0; k < n; ++k) key[k] = proj(x, y, (int32_t)k, sn, sd);
            for (int64_t k = 0; k < n; ++k) order[k] = (int32_t)k;
            qsort_r(order, (size_t)n, sizeof(int32_t), before_cmp, &oc);
            for (int64_t a = 0; a < n; ++a) pos[order[a]] = (int32_t)a;
            for (int64_t a = 0; a + h - 1 < n; ++a)
                score_window(x, y, order, h, a, sn, sd, pi, pj, &best);
            first = 0;
        }
        /* involved points and their positions */
        int64_t np = 0;
        for (size_t e = ga; e < gb; ++e) {
            int32_t pts[2] = { ev[e].i, ev[e].j };
            for (int q = 0; q < 2; ++q)
                if (!flag[pts[q]]) { flag[pts[q]] = 1; plist[np++] = pos[pts[q]]; }
        }
        qsort(plist, (size_t)np, sizeof(int32_t), cmp_i32);
        /* each involved position lies in a maximal run of equal projections;
         * re-sort every such run into the just-after order and re-score every
         * window with an end inside it */
        int64_t covered_to = -1;
        for (int64_t k = 0; k < np; ++k) {
            int64_t p = plist[k];
            if (p <= covered_to) continue;
            int64_t lo = p, hi = p;
            i128 kp = proj(x, y, order[p], sn, sd);
            while (lo > 0 && proj(x, y, order[lo - 1], sn, sd) == kp) --lo;
            while (hi + 1 < n && proj(x, y, order[hi + 1], sn, sd) == kp) ++hi;
            covered_to = hi;
            int64_t len = hi - lo + 1;
            memcpy(tmp, order + lo, sizeof(int32_t) * (size_t)len);
            qsort_r(tmp, (size_t)len, sizeof(int32_t), after_cmp, &oc);
            memcpy(order + lo, tmp, sizeof(int32_t) * (size_t)len);
            for (int64_t a = lo; a <= hi; ++a) pos[order[a]] = (int32_t)a;
            for (int64_t a = lo; a <= hi && a + h - 1 < n; ++a)
                score_window(x, y, order, h, a, sn, sd, pi, pj, &best);
            for (int64_t a = (lo - h + 1 > 0 ? lo - h + 1 : 0); a <= hi - h + 1; ++a)
                score_window(x, y, order, h, a, sn, sd, pi, pj, &best);
        }
        for (size_t e = ga; e < gb; ++e) { flag[ev[e].i] = 0; flag[ev[e].j] = 0; }
        ga = gb;
    }
    *best_out = best;
done:
    free(ev); free(order); free(pos); free(plist); free(tmp); free(flag); free(key);
    return rc;
}

/* --------------------------------------------------------------- drivers */

typedef int (*core_fn)(const int64_t *, const int64_t *, int64_t, int64_t, cand_t *);

static int run(core_fn fn, const int64_t *x, const int64_t *y, int64_t n, int64_t h,
               int scale_exp, oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 2 || !x || !y) { out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    if (h == 0) h = n / 2 + 1;
    if (h < 1 || h > n) { out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    cand_t best = {0};
    int rc = fn(x, y, n, h, &best);
    if (rc != OR_OK) { out->status = rc; return rc; }
    int status = OR_OK;
    if (!best.valid) {
        /* every x equal: no pairwise slope; report the window at slope 0 */
        i128 *keys = (i128 *)malloc(sizeof(i128) * (size_t)n);
        if (!keys) { out->status = OR_ERR_NOMEM; return OR_ERR_NOMEM; }
        eval_slope(x, y, n, h, 0, 1, keys, &best);
        free(keys);
        best.i = -1; best.j = -1;
        status = OR_ERR_VERTICAL;
    }
    finalize(&best, status, scale_exp, out);
    return status;
}

static int widen_i16(const int16_t *x, const int16_t *y, int64_t n, int64_t **X, int64_t **Y)
{
    *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    *Y = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!*X || !*Y) { free(*X); free(*Y); return OR_ERR_NOMEM; }
    for (int64_t k = 0; k < n; ++k) { (*X)[k] = x[k]; (*Y)[k] = y[k]; }
    return OR_OK;
}

/* Float32 values are exact dyadic rationals m * 2^e (|m| < 2^24); multiplying
 * every coordinate by 2^S, S = max over values of -e, makes all of them
 * integers without changing any slope; widths and intercepts scale by 2^S. */
static int widen_f32(const float *x, const float *y, int64_t n, int64_t **X, int64_t **Y,
                     int *S_out)
{
    int S = 0, emax = -100000;
    for (int64_t k = 0; k < 2 * n; ++k) {
        float v = k < n ? x[k] : y[k - n];
        if (!isfinite(v)) return OR_ERR_ARG;
        if (v == 0.0f) continue;
        int E;
        frexpf(v, &E);                 /* v = f * 2^E, 0.5 <= |f| < 1 */
        int e = E - 24;                /* v = (f * 2^24) * 2^e, f * 2^24 an integer */
        if (-e > S) S = -e;
        if (E > emax) emax = E;
    }
    if (emax != -100000 && emax + S > 60) return OR_ERR_UNSUPPORTED;
    *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    *Y = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!*X || !*Y) { free(*X); free(*Y); return OR_ERR_NOMEM; }
    for (int64_t k = 0; k < n; ++k) {
        (*X)[k] = (int64_t)ldexp((double)x[k], S);
        (*Y)[k] = (int64_t)ldexp((double)y[k], S);
    }
    *S_out = S;
    return OR_OK;
}

void oracle_set_threads(int t) { if (t > 0) omp_set_num_threads(t); }
int oracle_max_threads(void) { return omp_get_max_threads(); }

int oracle_lms_i16_brute(const int16_t *x, const int16_t *y, int64_t n, int64_t h,
                         oracle_result *out)
{
    int64_t *X, *Y;
    if (n < 2 || !x || !y) { memset(out, 0, sizeof(*out)); out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    if (widen_i16(x, y, n, &X, &Y)) { out->status = OR_ERR_NOMEM; return OR_ERR_NOMEM; }
    int rc = run(brute_core, X, Y, n, h, 0, out);
    free(X); free(Y);
    return rc;
}

int oracle_lms_i16_sweep(const int16_t *x, const int16_t *y, int64_t n, int64_t h,
                         oracle_result *out)
{
    int64_t *X, *Y;
    if (n < 2 || !x || !y) { memset(out, 0, sizeof(*out)); out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    if (widen_i16(x, y, n, &X, &Y)) { out->status = OR_ERR_NOMEM; return OR_ERR_NOMEM; }
    int rc = run(sweep_core, X, Y, n, h, 0, out);
    free(X); free(Y);
    return rc;
}

static int f32_entry(core_fn fn, const float *x, const float *y, int64_t n, int64_t h,
                     oracle_result *out)
{
    int64_t *X, *Y;
    int S = 0;
    memset(out, 0, sizeof(*out));
    if (n < 2 || !x || !y) { out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    int rc = widen_f32(x, y, n, &X, &Y, &S);
    if (rc) { out->status = rc; return rc; }
    rc = run(fn, X, Y, n, h, S, out);
    free(X); free(Y);
    return rc;
}

int oracle_lms_f32_brute(const float *x, const float *y, int64_t n, int64_t h,
                         oracle_result *out)
{
    return f32_entry(brute_core, x, y, n, h, out);
}

int oracle_lms_f32_sweep(const float *x, const float *y, int64_t n, int64_t h,
                         oracle_result *out)
{
    return f32_entry(sweep_core, x, y, n, h, out);
}

/* w(s) at one given slope s = sn/sd (sd > 0) for int16 points: the narrowest
 * window of h projections and its centre (used for certificates and bounds). */
int oracle_eval_slope_i16(const int16_t *x, const int16_t *y, int64_t n, int64_t h,
                          int64_t sn, int64_t sd, oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 1 || sd <= 0 || !x || !y) { out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    if (h == 0) h = n / 2 + 1;
    if (h < 1 || h > n) { out->status = OR_ERR_ARG; return OR_ERR_ARG; }
    int64_t *X, *Y;
    if (widen_i16(x, y, n, &X, &Y)) { out->status = OR_ERR_NOMEM; return OR_ERR_NOMEM; }
    i128 *keys = (i128 *)malloc(sizeof(i128) * (size_t)n);
    if (!keys) { free(X); free(Y); out->status = OR_ERR_NOMEM; return OR_ERR_NOMEM; }
    cand_t c;
    eval_slope(X, Y, n, h, sn, sd, keys, &c);
    c.i = -1; c.j = -1;
    finalize(&c, OR_OK, 0, out);
    free(keys); free(X); free(Y);
    return OR_OK;
}
