/*
 * FP64 CPU oracle for global (standard) Shepard inverse-distance weighting,
 * its gradients, the radius-limited and k-nearest-neighbour local forms
 * with their gradients, and modified Shepard weights on the radius form.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library.
 * It shares no code, header, table or helper with the CUDA library; the two
 * meet only through the seeded input generators.
 *
 * What it computes (Sec. 2.1, Eq. 1 of Mei & Tian, "Performance Impact of
 * Data Layout on the GPU-accelerated IDW Interpolation"):
 *
 *     Z(q) = sum_i w_i(q) z_i / sum_j w_j(q),    w_i(q) = d(q, x_i)^(-p)
 *
 * over ALL n data points (standard/global IDW, Sec. 1 and Sec. 2.1), with p
 * an arbitrary positive real (Sec. 2.1).
 *
 * Readings taken where the paper is silent:
 *   - d is the 2-D Euclidean distance in (x, y); the third coordinate of a
 *     data record is the sampled value z_i.
 *   - d^(-p) is evaluated as (d^2)^(-p/2); no square root is taken.
 *   - A query that coincides with a data point (d = 0, i.e. both coordinates
 *     numerically equal) returns z_i of the LOWEST such index i; Eq. 1 is
 *     undefined there.
 *   - Weights are scaled by the common factor (d2_min)^(p/2), where d2_min is
 *     the smallest squared distance of the query.  Eq. 1 is a ratio of two
 *     sums that are both homogeneous of degree one in the weights, so the
 *     factor cancels exactly; it keeps every weight in (0, 1] so that large
 *     p neither overflows nor underflows in FP64.
 *   - Both sums use Neumaier's compensated summation so that the oracle's own
 *     rounding error is far below the tolerances it is used to check.
 *   - NaN anywhere in a query's inputs gives NaN unless an exact hit is found.
 *
 * Local (radius-limited) variant (not the paper's method; the local Shepard
 * interpolation of its cited related work, Sec. 1): Eq. 1 over the data
 * points within distance R of the query only.  Readings:
 *   - membership is decided in FP32, exactly as a GPU evaluates it:
 *     dx = fl32(qx - x), dy = fl32(qy - y), d2 = fmaf(dy, dy, fl32(dx dx)),
 *     member iff d2 < fl32(R^2); the weights then use the exact FP64
 *     distances of the members;
 *   - an exact hit anywhere returns z of the lowest coincident index;
 *   - no member gives NaN;
 *   - data points with a non-finite coordinate are ignored (neither hits
 *     nor members);
 *   - its gradients hold each membership set fixed (the sets are piecewise
 *     constant in every input), so they are the global form's derivatives
 *     summed over the members; a query without members contributes none.
 *     The k-NN form's gradients hold each selection fixed the same way.
 *
 * k-nearest-neighbour variant (the other local form of the related work,
 * Sec. 1): Eq. 1 over the k data points nearest to the query.  Readings:
 *   - "nearest" ranks finite data points by the key (d2, index), d2 the same
 *     FP32 expression as the local membership test, so ties go to the lower
 *     index and both implementations select the same set;
 *   - the weights use the exact FP64 distances of the selected points;
 *   - an exact hit returns z of the lowest coincident index (the selection
 *     is still reported);
 *   - fewer than k finite points: all of them; none: NaN.
 *
 * Gradients (not in the paper; derived from Eq. 1 by the chain rule, with
 * S0 = sum w_i, S1 = sum w_i z_i, Z = S1/S0, w_i = (d_i^2)^(-p/2)):
 *   dZ/dz_i  = w_i / S0
 *   dZ/dq    = -(p/S0) sum_i (z_i - Z) w_i (q - x_i) / d_i^2
 *   dZ/dx_i  = +(p/S0)       (z_i - Z) w_i (q - x_i) / d_i^2
 *   dZ/dp    = -(1/(2 S0)) sum_i (z_i - Z) w_i ln d_i^2
 * At an exact hit Z = z_k, so dZ/dz_k = 1 and every other derivative is 0.
 * All of these ratios are unchanged by the common weight scaling above.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (no fast-math, no
 * contraction, so every operation is the plain IEEE double it reads as).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <unistd.h>

/* ------------------------------------------------------------------ sums */

typedef struct {
    double s; /* running sum */
    double c; /* Neumaier correction */
} nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_value(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------ one query */

static double sqdist(double qx, double qy, double x, double y)
{
    double dx = qx - x;
    double dy = qy - y;
    return dx * dx + dy * dy;
}

/* Scaled weight w_i / (d2_min)^(p/2) = (d2_min / d2)^(p/2). */
static double scaled_weight(double d2min, double d2, double p)
{
    double r = d2min / d2;
    if (p == 2.0)
        return r;
    return pow(r, 0.5 * p);
}

/*
 * Scans the data for an exact hit and the smallest squared distance.
 * Returns the lowest coincident index, or -1 if there is none.
 */
static int64_t scan_query(const double *data, int64_t n, double qx, double qy, double *d2min_out)
{
    double d2min = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double x = data[3 * i + 0];
        double y = data[3 * i + 1];
        if (x == qx && y == qy)
            return i;
        double d2 = sqdist(qx, qy, x, y);
        if (d2 < d2min)
            d2min = d2;
    }
    *d2min_out = d2min;
    return -1;
}

/*
 * Eq. 1 for one query.  Writes Z and the exact-hit index; optionally S0 and
 * Z's sums in the scaled form (S0 is the scaled weight sum, so S0 >= 1 when
 * there is no hit and the data are finite).
 */
static void one_query(const double *data, int64_t n, double qx, double qy, double p,
                      double *Z, int64_t *hit, double *S0_scaled, double *d2min_out)
{
    double d2min = 0.0;
    int64_t k = scan_query(data, n, qx, qy, &d2min);
    if (d2min_out)
        *d2min_out = d2min;
    if (k >= 0) {
        *Z = data[3 * k + 2];
        *hit = k;
        if (S0_scaled)
            *S0_scaled = INFINITY;
        return;
    }
    nsum s0 = {0.0, 0.0};
    nsum s1 = {0.0, 0.0};
    for (int64_t i = 0; i < n; i++) {
        double d2 = sqdist(qx, qy, data[3 * i + 0], data[3 * i + 1]);
        double w = scaled_weight(d2min, d2, p);
        nsum_add(&s0, w);
        nsum_add(&s1, w * data[3 * i + 2]);
    }
    double S0 = nsum_value(&s0);
    *Z = nsum_value(&s1) / S0;
    *hit = -1;
    if (S0_scaled)
        *S0_scaled = S0;
}

/* --------------------------------------------------------- thread pool */

typedef struct {
    void (*fn)(void *ctx, int64_t begin, int64_t end);
    void *ctx;
    int64_t begin, end;
} work;

static void *run_work(void *arg)
{
    work *w = (work *)arg;
    w->fn(w->ctx, w->begin, w->end);
    return NULL;
}

static int resolve_threads(int nthreads)
{
    if (nthreads > 0)
        return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* Runs fn over [0, count) split into contiguous ranges, one per thread. */
static int parallel_for(int64_t count, int nthreads,
                        void (*fn)(void *, int64_t, int64_t), void *ctx)
{
    int t = resolve_threads(nthreads);
    if ((int64_t)t > count)
        t = count > 0 ? (int)count : 1;
    pthread_t *tid = (pthread_t *)calloc((size_t)t, sizeof(pthread_t));
    work *ws = (work *)calloc((size_t)t, sizeof(work));
    if (!tid || !ws) {
        free(tid);
        free(ws);
        return -1;
    }
    for (int i = 0; i < t; i++) {
        ws[i].fn = fn;
        ws[i].ctx = ctx;
        ws[i].begin = count * i / t;
        ws[i].end = count * (i + 1) / t;
    }
    int started = 0;
    for (int i = 1; i < t; i++) {
        if (pthread_create(&tid[i], NULL, run_work, &ws[i]) != 0)
            break;
        started = i;
    }
    /* Ranges whose thread failed to start run here, sequentially. */
    run_work(&ws[0]);
    for (int i = started + 1; i < t; i++)
        run_work(&ws[i]);
    for (int i = 1; i <= started; i++)
        pthread_join(tid[i], NULL);
    free(tid);
    free(ws);
    return t;
}

/* ------------------------------------------------------------- forward */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    double p;
    double *Z;
    int64_t *hit;
    double *S0;
} fwd_ctx;

static void fwd_range(void *vctx, int64_t b, int64_t e)
{
    fwd_ctx *c = (fwd_ctx *)vctx;
    for (int64_t j = b; j < e; j++)
        one_query(c->data, c->n, c->q[2 * j], c->q[2 * j + 1], c->p, &c->Z[j], &c->hit[j],
                  c->S0 ? &c->S0[j] : NULL, NULL);
}

/*
 * Eq. 1 for m queries.
 *   data : n x 3 row-major doubles (x, y, z), host memory, caller-owned.
 *   q    : m x 2 row-major doubles (x, y).
 *   Z    : m doubles out.   hit : m int64 out (-1 = no exact hit).
 *   S0   : optional m doubles out, the scaled weight sum (inf at a hit).
 * Returns the number of threads used, or -1 on bad arguments.
 */
int oracle_idw_forward(const double *data, int64_t n, const double *q, int64_t m, double p,
                       double *Z, int64_t *hit, double *S0, int nthreads)
{
    if (!data || !q || !Z || !hit || n < 1 || m < 0 || !(p > 0.0) || !isfinite(p))
        return -1;
    fwd_ctx c = {data, n, q, p, Z, hit, S0};
    if (m == 0)
        return 0;
    return parallel_for(m, nthreads, fwd_range, &c);
}

/* ------------------------------------------------------- local variant */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    double p;
    float r2f; /* fl32(R^2) */
    double *Z;
    int64_t *hit;
    int32_t *count;
} local_ctx;

/* FP32 membership test: d2 = fmaf(dy, dy, fl32(dx dx)) < fl32(R^2). */
static int local_member(float qx, float qy, float x, float y, float r2f)
{
    float dx = qx - x;
    float dy = qy - y;
    float dxx = dx * dx;
    float d2 = fmaf(dy, dy, dxx);
    return d2 < r2f;
}

static void local_range(void *vctx, int64_t b, int64_t e)
{
    local_ctx *c = (local_ctx *)vctx;
    for (int64_t j = b; j < e; j++) {
        const double qx = c->q[2 * j], qy = c->q[2 * j + 1];
        const float qxf = (float)qx, qyf = (float)qy;
        int64_t k = -1;
        int32_t count = 0;
        double d2min = INFINITY;
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            if (!isfinite(x) || !isfinite(y))
                continue; /* ignored: neither a hit nor a member */
            if (x == qx && y == qy) {
                k = i;
                break;
            }
            if (local_member(qxf, qyf, (float)x, (float)y, c->r2f)) {
                const double d2 = sqdist(qx, qy, x, y);
                if (d2 < d2min)
                    d2min = d2;
                count++;
            }
        }
        c->hit[j] = k;
        if (k >= 0) {
            c->Z[j] = c->data[3 * k + 2];
            c->count[j] = -1;
            continue;
        }
        c->count[j] = count;
        if (count == 0) {
            c->Z[j] = NAN;
            continue;
        }
        nsum s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            if (!local_member(qxf, qyf, (float)x, (float)y, c->r2f))
                continue;
            const double w = scaled_weight(d2min, sqdist(qx, qy, x, y), c->p);
            nsum_add(&s0, w);
            nsum_add(&s1, w * c->data[3 * i + 2]);
        }
        c->Z[j] = nsum_value(&s1) / nsum_value(&s0);
    }
}

/*
 * Local Eq. 1: the data points within distance `radius` of each query.
 * Inputs as oracle_idw_forward (coordinates must be fp32 values); outputs
 * Z[m], hit[m] (lowest coincident index or -1) and count[m] (members used,
 * -1 at an exact hit).  Returns threads used, or -1 on bad arguments.
 */
int oracle_idw_local(const double *data, int64_t n, const double *q, int64_t m, double p,
                     double radius, double *Z, int64_t *hit, int32_t *count, int nthreads)
{
    if (!data || !q || !Z || !hit || !count || n < 1 || m < 0 || !(p > 0.0) || !isfinite(p) ||
        !(radius > 0.0))
        return -1;
    local_ctx c = {data, n, q, p, (float)(radius * radius), Z, hit, count};
    if (m == 0)
        return 0;
    return parallel_for(m, nthreads, local_range, &c);
}

/* ------------------------------------------------ local-form gradients */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    int64_t m;
    double p;
    float r2f;            /* fl32(R^2) */
    const double *g;      /* upstream gradient, m */
    double *Z;            /* m out */
    int64_t *hit;         /* m, pass A */
    int32_t *count;       /* m, pass A: members (-1 at a hit) */
    double *S0;           /* m, scaled by d2min^(p/2), pass A */
    double *d2min;        /* m, pass A: smallest member d^2 */
    double *grad_q;       /* m x 2 out */
    double *grad_p_part;  /* m out */
    double *grad_z;       /* n out */
    double *grad_xy;      /* n x 2 out */
} local_grad_ctx;

/*
 * Pass A of the local gradient, per query: the members, hit, Z and S0 exactly
 * as oracle_idw_local finds them, then dZ/dq and the query's share of dZ/dp,
 * the global formulas with every sum taken over the members only.
 */
static void local_grad_query_range(void *vctx, int64_t b, int64_t e)
{
    local_grad_ctx *c = (local_grad_ctx *)vctx;
    for (int64_t j = b; j < e; j++) {
        const double qx = c->q[2 * j], qy = c->q[2 * j + 1];
        const float qxf = (float)qx, qyf = (float)qy;
        int64_t hit = -1;
        int32_t members = 0;
        double dmin = INFINITY;
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            if (!isfinite(x) || !isfinite(y))
                continue;
            if (x == qx && y == qy) {
                hit = i;
                break;
            }
            if (local_member(qxf, qyf, (float)x, (float)y, c->r2f)) {
                const double d2 = sqdist(qx, qy, x, y);
                if (d2 < dmin)
                    dmin = d2;
                members++;
            }
        }
        c->hit[j] = hit;
        c->count[j] = hit >= 0 ? -1 : members;
        c->d2min[j] = dmin;
        c->grad_q[2 * j] = 0.0;
        c->grad_q[2 * j + 1] = 0.0;
        c->grad_p_part[j] = 0.0;
        if (hit >= 0) { /* exact hit: z of that point, no coordinate gradient */
            c->Z[j] = c->data[3 * hit + 2];
            continue;
        }
        if (members == 0) {
            c->Z[j] = NAN; /* no neighbourhood: no value and no gradient */
            continue;
        }
        nsum s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            const int member = local_member(qxf, qyf, (float)x, (float)y, c->r2f);
            if (!member)
                continue;
            const double w = scaled_weight(dmin, sqdist(qx, qy, x, y), c->p);
            nsum_add(&s0, w);
            nsum_add(&s1, w * c->data[3 * i + 2]);
        }
        const double S0 = nsum_value(&s0), Zj = nsum_value(&s1) / S0;
        c->S0[j] = S0;
        c->Z[j] = Zj;
        nsum sx = {0, 0}, sy = {0, 0}, sp = {0, 0};
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            const int member = local_member(qxf, qyf, (float)x, (float)y, c->r2f);
            if (!member)
                continue; /* members only: the query-side sums */
            const double dx = qx - x, dy = qy - y, d2 = dx * dx + dy * dy;
            const double w = scaled_weight(dmin, d2, c->p);
            const double a = (c->data[3 * i + 2] - Zj) * w;
            nsum_add(&sx, a * dx / d2);
            nsum_add(&sy, a * dy / d2);
            nsum_add(&sp, a * log(d2));
        }
        const double gj = c->g[j];
        c->grad_q[2 * j] = -gj * (c->p / S0) * nsum_value(&sx);
        c->grad_q[2 * j + 1] = -gj * (c->p / S0) * nsum_value(&sy);
        c->grad_p_part[j] = -0.5 * gj * nsum_value(&sp) / S0;
    }
}

/* Pass B, per data point: the sums over the queries whose neighbourhood
 * holds it of dZ/dz_i and dZ/dx_i (an exact hit passes g_j to its point). */
static void local_grad_data_range(void *vctx, int64_t b, int64_t e)
{
    local_grad_ctx *c = (local_grad_ctx *)vctx;
    for (int64_t i = b; i < e; i++) {
        const double x = c->data[3 * i], y = c->data[3 * i + 1], z = c->data[3 * i + 2];
        const float xf = (float)x, yf = (float)y;
        nsum tz = {0, 0}, tx = {0, 0}, ty = {0, 0};
        for (int64_t j = 0; j < c->m; j++) {
            const double gj = c->g[j];
            if (c->hit[j] >= 0) {
                if (c->hit[j] == i)
                    nsum_add(&tz, gj); /* dZ/dz at a hit */
                continue;
            }
            if (c->count[j] == 0)
                continue;
            const double qx = c->q[2 * j], qy = c->q[2 * j + 1];
            if (!local_member((float)qx, (float)qy, xf, yf, c->r2f))
                continue; /* i is outside query j's neighbourhood */
            const double dx = qx - x, dy = qy - y, d2 = dx * dx + dy * dy;
            const double w = scaled_weight(c->d2min[j], d2, c->p);
            const double S0 = c->S0[j];
            nsum_add(&tz, gj * w / S0);
            const double a = gj * (c->p / S0) * (z - c->Z[j]) * w / d2;
            nsum_add(&tx, a * dx);
            nsum_add(&ty, a * dy);
        }
        c->grad_z[i] = nsum_value(&tz);
        c->grad_xy[2 * i] = nsum_value(&tx);
        c->grad_xy[2 * i + 1] = nsum_value(&ty);
    }
}

/*
 * Gradient of L = sum_j g_j Z(q_j) for the local form (oracle_idw_local):
 * the membership sets are held fixed (they are piecewise constant in every
 * input), so each derivative is the global one summed over the members.  A
 * query with an exact hit passes g_j to dL/dz of the hit point and nothing
 * else; a query with no member contributes nothing.
 *   data, q, p, radius : as oracle_idw_local.   g : m doubles.
 *   Outputs (host memory): Z[m], grad_z[n], grad_xy[n x 2], grad_q[m x 2],
 *   grad_p[1].
 * Returns the number of threads used, or -1 on bad arguments / no memory.
 */
int oracle_idw_local_grad(const double *data, int64_t n, const double *q, int64_t m, double p,
                          double radius, const double *g, double *Z, double *grad_z,
                          double *grad_xy, double *grad_q, double *grad_p, int nthreads)
{
    if (!data || !q || !g || !Z || !grad_z || !grad_xy || !grad_q || !grad_p || n < 1 ||
        m < 1 || !(p > 0.0) || !isfinite(p) || !(radius > 0.0))
        return -1;
    int64_t *hit = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int32_t *count = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    double *S0 = (double *)malloc((size_t)m * sizeof(double));
    double *d2min = (double *)malloc((size_t)m * sizeof(double));
    double *gp = (double *)malloc((size_t)m * sizeof(double));
    int t = -1;
    if (hit && count && S0 && d2min && gp) {
        local_grad_ctx c = {data, n, q, m, p, (float)(radius * radius), g, Z, hit, count,
                            S0, d2min, grad_q, gp, grad_z, grad_xy};
        t = parallel_for(m, nthreads, local_grad_query_range, &c);
        if (t > 0)
            t = parallel_for(n, nthreads, local_grad_data_range, &c);
        nsum total = {0, 0};
        for (int64_t j = 0; j < m; j++)
            nsum_add(&total, gp[j]);
        *grad_p = nsum_value(&total);
    }
    free(hit);
    free(count);
    free(S0);
    free(d2min);
    free(gp);
    return t;
}

/* ------------------------------------------- modified Shepard variant */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    double p;
    double radius;
    float r2f; /* fl32(R^2) */
    double *Z;
    int64_t *hit;
    int32_t *count;
} modified_ctx;

/* The modified Shepard weight's base t = (R - d) / (R d) = 1/d - 1/R of a
 * member, taken as 0 where exact arithmetic puts the point at or beyond R
 * (the FP32 membership test can admit such points). */
static double modified_base(double radius, double d)
{
    const double t = isinf(radius) ? 1.0 / d : (radius - d) / (radius * d);
    return t > 0.0 ? t : 0.0;
}

static void modified_range(void *vctx, int64_t b, int64_t e)
{
    modified_ctx *c = (modified_ctx *)vctx;
    for (int64_t j = b; j < e; j++) {
        const double qx = c->q[2 * j], qy = c->q[2 * j + 1];
        const float qxf = (float)qx, qyf = (float)qy;
        int64_t k = -1;
        int32_t members = 0;
        double tmax = 0.0;
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            if (!isfinite(x) || !isfinite(y))
                continue;
            if (x == qx && y == qy) {
                k = i;
                break;
            }
            if (local_member(qxf, qyf, (float)x, (float)y, c->r2f)) {
                const double t = modified_base(c->radius, sqrt(sqdist(qx, qy, x, y)));
                if (t > tmax)
                    tmax = t;
                members++;
            }
        }
        c->hit[j] = k;
        if (k >= 0) {
            c->Z[j] = c->data[3 * k + 2];
            c->count[j] = -1;
            continue;
        }
        c->count[j] = members;
        if (members == 0 || tmax == 0.0) { /* no member with a positive weight */
            c->Z[j] = NAN;
            continue;
        }
        /* Weights relative to the largest, (t_i / t_max)^p in (0, 1]. */
        nsum m0 = {0.0, 0.0}, m1 = {0.0, 0.0};
        for (int64_t i = 0; i < c->n; i++) {
            const double x = c->data[3 * i], y = c->data[3 * i + 1];
            const int inside = local_member(qxf, qyf, (float)x, (float)y, c->r2f);
            if (!inside)
                continue;
            const double t = modified_base(c->radius, sqrt(sqdist(qx, qy, x, y)));
            const double w = pow(t / tmax, c->p);
            nsum_add(&m0, w);
            nsum_add(&m1, w * c->data[3 * i + 2]);
        }
        c->Z[j] = nsum_value(&m1) / nsum_value(&m0);
    }
}

/*
 * Modified Shepard interpolation (Franke & Nielson's local weights, a local
 * variant in the family of the paper's related work, Sec. 1): Eq. 1 over
 * the members of the radius form (the same FP32 test), with the weights
 *     w_i = ((R - d_i) / (R d_i))^p = (1/d_i - 1/R)^p,
 * which fall to 0 continuously at d = R.  R = +inf gives d^-p, the global
 * form.  Exact hit: z of the lowest coincident index (count -1); no member
 * with a positive weight: NaN.  Outputs and return as oracle_idw_local.
 */
int oracle_idw_modified(const double *data, int64_t n, const double *q, int64_t m, double p,
                        double radius, double *Z, int64_t *hit, int32_t *count, int nthreads)
{
    if (!data || !q || !Z || !hit || !count || n < 1 || m < 0 || !(p > 0.0) || !isfinite(p) ||
        !(radius > 0.0))
        return -1;
    modified_ctx c = {data, n, q, p, radius, (float)(radius * radius), Z, hit, count};
    if (m == 0)
        return 0;
    return parallel_for(m, nthreads, modified_range, &c);
}

/* Gradient of L = sum_j g_j Z(q_j) for modified Shepard (oracle_idw_modified),
 * membership held fixed as for the radius form.  With t_i = 1/d_i - 1/R and
 * w_i = t_i^p (scaled by t_max^p, which cancels):
 *     dw_i/dq = -p w_i (q - x_i) / (t_i d_i^3) = -dw_i/dx_i,   dw_i/dp = w_i ln t_i,
 * so dZ/dq = -(p/S0) sum_i (z_i - Z) w_i (q - x_i)/(t_i d_i^3), dZ/dx_i the
 * negated term, dZ/dz_i = w_i/S0 and dZ/dp = (1/S0) sum_i (z_i - Z) w_i ln t_i.
 * Members of zero weight (t_i = 0) contribute nothing.  Hits and empty
 * neighbourhoods as oracle_idw_local_grad.  Returns threads used (1), or -1. */
int oracle_idw_modified_grad(const double *data, int64_t n, const double *q, int64_t m, double p,
                             double radius, const double *g, double *Z, double *grad_z,
                             double *grad_xy, double *grad_q, double *grad_p)
{
    if (!data || !q || !g || !Z || !grad_z || !grad_xy || !grad_q || !grad_p || n < 1 ||
        m < 1 || !(p > 0.0) || !isfinite(p) || !(radius > 0.0))
        return -1;
    int64_t *hit = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int32_t *count = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    nsum *acc = (nsum *)calloc((size_t)n * 3, sizeof(nsum)); /* per point: z, x, y */
    int t = -1;
    if (hit && count && acc)
        t = oracle_idw_modified(data, n, q, m, p, radius, Z, hit, count, 1);
    const float r2f = (float)(radius * radius);
    if (t >= 0) {
        nsum ptot = {0, 0};
        for (int64_t j = 0; j < m; j++) {
            const double gj = g[j], qx = q[2 * j], qy = q[2 * j + 1];
            const float qxf = (float)qx, qyf = (float)qy;
            grad_q[2 * j] = 0.0;
            grad_q[2 * j + 1] = 0.0;
            if (hit[j] >= 0) { /* exact hit: all of g_j goes to the point's z */
                nsum_add(&acc[3 * hit[j]], gj);
                continue;
            }
            if (isnan(Z[j]))
                continue;
            double tm = 0.0;
            for (int64_t i = 0; i < n; i++) {
                const double *x = data + 3 * i;
                if (local_member(qxf, qyf, (float)x[0], (float)x[1], r2f)) {
                    const double tt = modified_base(radius, sqrt(sqdist(qx, qy, x[0], x[1])));
                    if (tt > tm)
                        tm = tt;
                }
            }
            nsum u0 = {0, 0};
            for (int64_t i = 0; i < n; i++) {
                const double *x = data + 3 * i;
                if (local_member(qxf, qyf, (float)x[0], (float)x[1], r2f))
                    nsum_add(&u0, pow(modified_base(radius, sqrt(sqdist(qx, qy, x[0], x[1]))) / tm, p));
            }
            const double S0 = nsum_value(&u0), Zj = Z[j];
            nsum vx = {0, 0}, vy = {0, 0}, vp = {0, 0};
            for (int64_t i = 0; i < n; i++) {
                const double *x = data + 3 * i;
                if (!local_member(qxf, qyf, (float)x[0], (float)x[1], r2f))
                    continue;
                const double ex = qx - x[0], ey = qy - x[1], d = sqrt(ex * ex + ey * ey);
                const double tt = modified_base(radius, d);
                if (tt == 0.0)
                    continue; /* zero weight: no derivative either */
                const double w = pow(tt / tm, p);
                const double b = (x[2] - Zj) * w;
                const double f = b / (tt * d * d * d); /* (z_i - Z) w_i / (t_i d_i^3) */
                nsum_add(&vx, f * ex);
                nsum_add(&vy, f * ey);
                nsum_add(&vp, b * log(tt));
                nsum_add(&acc[3 * i], gj * w / S0);
                nsum_add(&acc[3 * i + 1], gj * (p / S0) * f * ex);
                nsum_add(&acc[3 * i + 2], gj * (p / S0) * f * ey);
            }
            grad_q[2 * j] = -gj * (p / S0) * nsum_value(&vx);
            grad_q[2 * j + 1] = -gj * (p / S0) * nsum_value(&vy);
            nsum_add(&ptot, gj * nsum_value(&vp) / S0);
        }
        for (int64_t i = 0; i < n; i++) {
            grad_z[i] = nsum_value(&acc[3 * i]);
            grad_xy[2 * i] = nsum_value(&acc[3 * i + 1]);
            grad_xy[2 * i + 1] = nsum_value(&acc[3 * i + 2]);
        }
        *grad_p = nsum_value(&ptot);
    }
    free(hit);
    free(count);
    free(acc);
    return t;
}

/* ------------------------------------------------------- k-NN variant */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    double p;
    int k;
    double *Z;
    int64_t *hit;
    float *kd2;
    int64_t *nbr;
    int32_t *count;
} knn_ctx;

static float fp32_d2(float qx, float qy, float x, float y)
{
    float dx = qx - x;
    float dy = qy - y;
    float dxx = dx * dx;
    return fmaf(dy, dy, dxx);
}

/* Key order: smaller d2 first, then smaller index. */
static int key_less(float da, int64_t ia, float db, int64_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* Max-heap on the key, size `size`, stored in (hd, hi). */
static void heap_sift_down(float *hd, int64_t *hi, int size, int at)
{
    for (;;) {
        int l = 2 * at + 1, r = l + 1, big = at;
        if (l < size && key_less(hd[big], hi[big], hd[l], hi[l]))
            big = l;
        if (r < size && key_less(hd[big], hi[big], hd[r], hi[r]))
            big = r;
        if (big == at)
            return;
        float td = hd[at];
        int64_t ti = hi[at];
        hd[at] = hd[big];
        hi[at] = hi[big];
        hd[big] = td;
        hi[big] = ti;
        at = big;
    }
}

static void heap_sift_up(float *hd, int64_t *hi, int at)
{
    while (at > 0) {
        int parent = (at - 1) / 2;
        if (!key_less(hd[parent], hi[parent], hd[at], hi[at]))
            return;
        float td = hd[at];
        int64_t ti = hi[at];
        hd[at] = hd[parent];
        hi[at] = hi[parent];
        hd[parent] = td;
        hi[parent] = ti;
        at = parent;
    }
}

static void knn_range(void *vctx, int64_t b, int64_t e)
{
    knn_ctx *c = (knn_ctx *)vctx;
    const int k = c->k;
    float *hd = (float *)malloc(sizeof(float) * (size_t)k);
    int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!hd || !hi) {
        free(hd);
        free(hi);
        for (int64_t j = b; j < e; j++)
            c->Z[j] = NAN, c->count[j] = -2;
        return;
    }
    for (int64_t j = b; j < e; j++) {
        const double qx = c->q[2 * j], qy = c->q[2 * j + 1];
        const float qxf = (float)qx, qyf = (float)qy;
        int64_t hit = -1;
        int size = 0;
        if (isfinite(qx) && isfinite(qy)) {
            for (int64_t i = 0; i < c->n; i++) {
                const double x = c->data[3 * i], y = c->data[3 * i + 1];
                if (!isfinite(x) || !isfinite(y))
                    continue;
                if (hit < 0 && x == qx && y == qy)
                    hit = i;
                const float d2 = fp32_d2(qxf, qyf, (float)x, (float)y);
                if (size < k) {
                    hd[size] = d2;
                    hi[size] = i;
                    heap_sift_up(hd, hi, size);
                    size++;
                } else if (key_less(d2, i, hd[0], hi[0])) {
                    hd[0] = d2;
                    hi[0] = i;
                    heap_sift_down(hd, hi, size, 0);
                }
            }
        }
        /* Report the selection in key order (heap sort, ascending). */
        int64_t *out = c->nbr + (size_t)j * (size_t)k;
        for (int t = 0; t < k; t++)
            out[t] = -1;
        c->kd2[j] = size > 0 ? hd[0] : NAN;
        for (int s = size; s > 0; s--) {
            out[s - 1] = hi[0];
            hd[0] = hd[s - 1];
            hi[0] = hi[s - 1];
            heap_sift_down(hd, hi, s - 1, 0);
        }
        c->hit[j] = hit;
        c->count[j] = size;
        if (hit >= 0) {
            c->Z[j] = c->data[3 * hit + 2];
            continue;
        }
        if (size == 0) {
            c->Z[j] = NAN;
            continue;
        }
        double d2min = INFINITY;
        for (int t = 0; t < size; t++) {
            const int64_t i = out[t];
            const double d2 = sqdist(qx, qy, c->data[3 * i], c->data[3 * i + 1]);
            if (d2 < d2min)
                d2min = d2;
        }
        nsum s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
        for (int t = 0; t < size; t++) {
            const int64_t i = out[t];
            const double w = scaled_weight(d2min, sqdist(qx, qy, c->data[3 * i], c->data[3 * i + 1]),
                                           c->p);
            nsum_add(&s0, w);
            nsum_add(&s1, w * c->data[3 * i + 2]);
        }
        c->Z[j] = nsum_value(&s1) / nsum_value(&s0);
    }
    free(hd);
    free(hi);
}

/*
 * k-NN Eq. 1: the k data points nearest to each query by the key
 * (fl32 d2, index).  Outputs Z[m], hit[m] (lowest coincident index or -1),
 * kd2[m] (the FP32 d2 of the last selected point, NaN if none), nbr[m*k]
 * (selected indices in key order, -1 padded) and count[m] (points
 * selected: min(k, finite points), 0 for a non-finite query).  Returns
 * threads used, or -1 on bad arguments.
 */
int oracle_idw_knn(const double *data, int64_t n, const double *q, int64_t m, double p, int k,
                   double *Z, int64_t *hit, float *kd2, int64_t *nbr, int32_t *count,
                   int nthreads)
{
    if (!data || !q || !Z || !hit || !kd2 || !nbr || !count || n < 1 || m < 0 || k < 1 ||
        !(p > 0.0) || !isfinite(p))
        return -1;
    knn_ctx c = {data, n, q, p, k, Z, hit, kd2, nbr, count};
    if (m == 0)
        return 0;
    return parallel_for(m, nthreads, knn_range, &c);
}

/* ------------------------------------------------------------ gradients */

typedef struct {
    const double *data;
    int64_t n;
    const double *q;
    int64_t m;
    double p;
    const double *g;      /* upstream gradient, m */
    double *Z;            /* m, from pass A */
    int64_t *hit;         /* m, from pass A */
    double *S0;           /* m, scaled, from pass A */
    double *d2min;        /* m, from pass A */
    double *grad_q;       /* m x 2 out */
    double *grad_p_part;  /* m out: per-query share of dL/dp */
    double *grad_z;       /* n out */
    double *grad_xy;      /* n x 2 out */
} grad_ctx;

/* Pass A: per query, Z, S0, and the query-side sums of dZ/dq and dZ/dp. */
static void grad_query_range(void *vctx, int64_t b, int64_t e)
{
    grad_ctx *c = (grad_ctx *)vctx;
    for (int64_t j = b; j < e; j++) {
        double qx = c->q[2 * j], qy = c->q[2 * j + 1];
        one_query(c->data, c->n, qx, qy, c->p, &c->Z[j], &c->hit[j], &c->S0[j], &c->d2min[j]);
        if (c->hit[j] >= 0) {
            c->grad_q[2 * j] = 0.0;
            c->grad_q[2 * j + 1] = 0.0;
            c->grad_p_part[j] = 0.0;
            continue;
        }
        nsum gx = {0, 0}, gy = {0, 0}, gp = {0, 0};
        for (int64_t i = 0; i < c->n; i++) {
            double x = c->data[3 * i], y = c->data[3 * i + 1], z = c->data[3 * i + 2];
            double dx = qx - x, dy = qy - y;
            double d2 = dx * dx + dy * dy;
            double w = scaled_weight(c->d2min[j], d2, c->p);
            double a = (z - c->Z[j]) * w;
            nsum_add(&gx, a * dx / d2);
            nsum_add(&gy, a * dy / d2);
            nsum_add(&gp, a * log(d2));
        }
        double gj = c->g[j];
        double S0 = c->S0[j];
        c->grad_q[2 * j] = -gj * (c->p / S0) * nsum_value(&gx);
        c->grad_q[2 * j + 1] = -gj * (c->p / S0) * nsum_value(&gy);
        c->grad_p_part[j] = -gj * nsum_value(&gp) / (2.0 * S0);
    }
}

/* Pass B: per data point, the sums over queries of dZ/dz_i and dZ/dx_i. */
static void grad_data_range(void *vctx, int64_t b, int64_t e)
{
    grad_ctx *c = (grad_ctx *)vctx;
    for (int64_t i = b; i < e; i++) {
        double x = c->data[3 * i], y = c->data[3 * i + 1], z = c->data[3 * i + 2];
        nsum gz = {0, 0}, gx = {0, 0}, gy = {0, 0};
        for (int64_t j = 0; j < c->m; j++) {
            double gj = c->g[j];
            if (c->hit[j] >= 0) {
                if (c->hit[j] == i)
                    nsum_add(&gz, gj);
                continue;
            }
            double qx = c->q[2 * j], qy = c->q[2 * j + 1];
            double dx = qx - x, dy = qy - y;
            double d2 = dx * dx + dy * dy;
            double w = scaled_weight(c->d2min[j], d2, c->p);
            double S0 = c->S0[j];
            nsum_add(&gz, gj * w / S0);
            double a = gj * (c->p / S0) * (z - c->Z[j]) * w / d2;
            nsum_add(&gx, a * dx);
            nsum_add(&gy, a * dy);
        }
        c->grad_z[i] = nsum_value(&gz);
        c->grad_xy[2 * i] = nsum_value(&gx);
        c->grad_xy[2 * i + 1] = nsum_value(&gy);
    }
}

/*
 * Gradient of L = sum_j g_j Z(q_j) with respect to every input of Eq. 1.
 *   data, q, p : as in oracle_idw_forward.   g : m doubles (dL/dZ_j).
 *   Outputs (all required, host memory): Z[m], grad_z[n], grad_xy[n x 2],
 *   grad_q[m x 2], grad_p[1].
 * Returns the number of threads used, or -1 on bad arguments / no memory.
 */
int oracle_idw_grad(const double *data, int64_t n, const double *q, int64_t m, double p,
                    const double *g, double *Z, double *grad_z, double *grad_xy,
                    double *grad_q, double *grad_p, int nthreads)
{
    if (!data || !q || !g || !Z || !grad_z || !grad_xy || !grad_q || !grad_p || n < 1 ||
        m < 1 || !(p > 0.0) || !isfinite(p))
        return -1;
    int64_t *hit = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    double *S0 = (double *)malloc((size_t)m * sizeof(double));
    double *d2min = (double *)malloc((size_t)m * sizeof(double));
    double *gp = (double *)malloc((size_t)m * sizeof(double));
    if (!hit || !S0 || !d2min || !gp) {
        free(hit);
        free(S0);
        free(d2min);
        free(gp);
        return -1;
    }
    grad_ctx c = {data, n, q, m, p, g, Z, hit, S0, d2min, grad_q, gp, grad_z, grad_xy};
    int t = parallel_for(m, nthreads, grad_query_range, &c);
    if (t > 0)
        t = parallel_for(n, nthreads, grad_data_range, &c);
    nsum total = {0, 0};
    for (int64_t j = 0; j < m; j++)
        nsum_add(&total, gp[j]);
    *grad_p = nsum_value(&total);
    free(hit);
    free(S0);
    free(d2min);
    free(gp);
    return t;
}

/* -------------------------------------------------- k-NN gradients */

/*
 * Gradient of L = sum_j g_j Z(q_j) for the k-NN form (oracle_idw_knn): each
 * query's selection, the k smallest keys (fl32 d2, index), is held fixed (it
 * is piecewise constant in every input), so each derivative is the global
 * one summed over the selected points.  A query with an exact hit passes
 * g_j to dL/dz of the hit point and nothing else; a query that selects
 * nothing contributes nothing.  Arguments as oracle_idw_local_grad, with k
 * in place of the radius.  The selection runs on `nthreads` threads, the
 * gradient sums on one.  Returns threads used, or -1 on bad arguments / no
 * memory.
 */
int oracle_idw_knn_grad(const double *data, int64_t n, const double *q, int64_t m, double p,
                        int k, const double *g, double *Z, double *grad_z, double *grad_xy,
                        double *grad_q, double *grad_p, int nthreads)
{
    if (!data || !q || !g || !Z || !grad_z || !grad_xy || !grad_q || !grad_p || n < 1 ||
        m < 1 || k < 1 || !(p > 0.0) || !isfinite(p))
        return -1;
    int64_t *hit = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    float *kd2 = (float *)malloc((size_t)m * sizeof(float));
    int64_t *nbr = (int64_t *)malloc((size_t)m * (size_t)k * sizeof(int64_t));
    int32_t *count = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    nsum *acc = (nsum *)calloc((size_t)n * 3, sizeof(nsum)); /* per point: z, x, y */
    int t = -1;
    if (hit && kd2 && nbr && count && acc)
        t = oracle_idw_knn(data, n, q, m, p, k, Z, hit, kd2, nbr, count, nthreads);
    if (t >= 0) {
        nsum ptot = {0, 0};
        for (int64_t j = 0; j < m; j++) {
            const double gj = g[j], qx = q[2 * j], qy = q[2 * j + 1];
            const int64_t *sel = nbr + j * (int64_t)k;
            grad_q[2 * j] = 0.0;
            grad_q[2 * j + 1] = 0.0;
            if (hit[j] >= 0) { /* the hit point takes the whole of g_j */
                nsum_add(&acc[3 * hit[j]], gj);
                continue;
            }
            const int cnt = count[j];
            if (cnt <= 0)
                continue;
            double dmin = INFINITY;
            for (int s = 0; s < cnt; s++) {
                const double d2 = sqdist(qx, qy, data[3 * sel[s]], data[3 * sel[s] + 1]);
                if (d2 < dmin)
                    dmin = d2;
            }
            nsum w0 = {0, 0}, w1 = {0, 0};
            for (int s = 0; s < cnt; s++) {
                const double *x = data + 3 * sel[s];
                const double w = scaled_weight(dmin, sqdist(qx, qy, x[0], x[1]), p);
                nsum_add(&w0, w);
                nsum_add(&w1, w * x[2]);
            }
            const double S0 = nsum_value(&w0), Zj = nsum_value(&w1) / S0;
            nsum qsx = {0, 0}, qsy = {0, 0}, qsp = {0, 0};
            for (int s = 0; s < cnt; s++) {
                const double *x = data + 3 * sel[s];
                const double ex = qx - x[0], ey = qy - x[1], e2 = ex * ex + ey * ey;
                const double w = scaled_weight(dmin, e2, p);
                const double b = (x[2] - Zj) * w; /* (z_i - Z) w_i */
                nsum_add(&qsx, b * ex / e2);
                nsum_add(&qsy, b * ey / e2);
                nsum_add(&qsp, b * log(e2));
                nsum_add(&acc[3 * sel[s]], gj * w / S0);
                const double f = gj * (p / S0) * b / e2;
                nsum_add(&acc[3 * sel[s] + 1], f * ex);
                nsum_add(&acc[3 * sel[s] + 2], f * ey);
            }
            grad_q[2 * j] = -gj * (p / S0) * nsum_value(&qsx);
            grad_q[2 * j + 1] = -gj * (p / S0) * nsum_value(&qsy);
            nsum_add(&ptot, -gj * nsum_value(&qsp) / (2.0 * S0));
        }
        for (int64_t i = 0; i < n; i++) {
            grad_z[i] = nsum_value(&acc[3 * i]);
            grad_xy[2 * i] = nsum_value(&acc[3 * i + 1]);
            grad_xy[2 * i + 1] = nsum_value(&acc[3 * i + 2]);
        }
        *grad_p = nsum_value(&ptot);
    }
    free(hit);
    free(kd2);
    free(nbr);
    free(count);
    free(acc);
    return t;
}

