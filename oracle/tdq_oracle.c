/*
 * tdq_oracle.c -- plain CPU FP64 oracle for the distance threshold search of
 * Gowanlock & Casanova, "Parallel Distance Threshold Query Processing for
 * Spatiotemporal Trajectory Databases on the GPU" (arXiv 1405.7461).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library under paper_1405_7461_gb300/csrc) shares no code with it:
 * no headers, no helpers, no constants.
 *
 * What it computes (Sec. 3, Problem Definition): the database D holds n
 * 4-D line segments, each given by a start point (x,y,z,t_start) and an end
 * point (x,y,z,t_end); a query Q is a set of such segments.  For every
 * (query segment, entry segment) pair it reports the sub-interval of time,
 * inside the query window [t0,t1], during which the two moving points are
 * within distance d of each other, when that sub-interval is not empty.
 *
 * Per pair it follows the two steps named in Sec. 5 / Algorithm 1:
 *   temporalIntersection -- clip both segments to their common time span by
 *                           linear interpolation, and
 *   calcTimeInterval     -- the time interval where the clipped segments are
 *                           within d, found from a degree-two polynomial.
 * Readings taken where the paper is silent:
 *   - pairs whose common span has zero length are not reported (a < b strict);
 *   - "within d" is inclusive (distance <= d);
 *   - the window [t0,t1] clips the common span like the segments do;
 *   - the decision "interval non-empty" is taken on the distance of closest
 *     approach inside the span, evaluated directly at the closest point;
 *   - the roots use the cancellation-free quadratic formula (Numerical
 *     Recipes, Sec. 5.6).
 *
 * Search drivers:
 *   oracle_search_bruteforce -- every query segment against every entry.
 *   oracle_search_sweep      -- the same per-pair function, but entries are
 *                               first sorted by t_start and only those whose
 *                               start lies in (q.t_start - maxdur, q.t_end)
 *                               are visited (pruning only; identical result).
 *   oracle_search_sweep_per_query -- the sweep with a threshold and window
 *                               of its own for every query segment.
 *   oracle_self_join         -- the sweep with the database as the query
 *                               set, pairs of one trajectory left out and
 *                               each unordered pair reported once (query (ii)
 *                               of Sec. 2.1).
 * And the temporal-bin index of Sec. 4 (Fig. 1) plus the interaction count of
 * a query batching over it (Fig. 2), for the index pins.
 *
 * Compiled with -O2 -ffp-contract=off so that no multiply-add is fused and the
 * arithmetic is the same on every host.
 *
 * ORACLE_MUTANT (undefined in every normal build) plants one deliberate
 * mistake, so that the test-suite can show that its pins catch it.
 */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* One segment, as defined in Sec. 3: start point, end point.                */
typedef struct {
    double x0, y0, z0, t0; /* start */
    double x1, y1, z1, t1; /* end   */
} oseg;

static oseg load_seg(const double *const *a, int64_t i)
{
    oseg s;
    s.x0 = a[0][i]; s.y0 = a[1][i]; s.z0 = a[2][i]; s.t0 = a[3][i];
    s.x1 = a[4][i]; s.y1 = a[5][i]; s.z1 = a[6][i]; s.t1 = a[7][i];
    return s;
}

/* Position of the moving point of segment s at time t (t inside its extent):
 * straight-line interpolation between its two endpoints (Sec. 3). */
static void position_at(const oseg *s, double t, double p[3])
{
    double f = (t - s->t0) / (s->t1 - s->t0);
    if (ORACLE_MUTANT == 3) f = (s->t1 - t) / (s->t1 - s->t0);
    p[0] = s->x0 + (s->x1 - s->x0) * f;
    p[1] = s->y0 + (s->y1 - s->y0) * f;
    p[2] = s->z0 + (s->z1 - s->z0) * f;
}

static double dmax3(double a, double b, double c)
{
    double m = a > b ? a : b;
    return m > c ? m : c;
}
static double dmin3(double a, double b, double c)
{
    double m = a < b ? a : b;
    return m < c ? m : c;
}

/*
 * The per-pair computation (Sec. 5, Algorithm 1: temporalIntersection then
 * calcTimeInterval).
 *
 * Returns -1 when the two segments have no common time span of positive
 * length inside [wt0, wt1]; 0 when they share a span but never come within
 * d of each other in it; 1 when they do, with the interval [*t_enter,
 * *t_exit] in absolute time.  *dmin receives the distance of closest
 * approach inside the span whenever the return value is >= 0.
 */
int oracle_pair(const double e8[8], const double q8[8], double d, double wt0, double wt1,
                double *t_enter, double *t_exit, double *dmin)
{
    oseg e, q;
    memcpy(&e, e8, sizeof e);
    memcpy(&q, q8, sizeof q);

    /* temporalIntersection: the common span [a, b]. */
    double a = dmax3(e.t0, q.t0, wt0);
    double b = dmin3(e.t1, q.t1, wt1);
    if (ORACLE_MUTANT == 8) {
        a = dmax3(e.t0, q.t0, -INFINITY);
        b = dmin3(e.t1, q.t1, INFINITY);
    }
    if (ORACLE_MUTANT == 4 ? !(a <= b) : !(a < b))
        return -1;

    /* Both segments clipped to [a, b]: their endpoints at a and at b. */
    double ea[3], eb[3], qa[3], qb[3];
    position_at(&e, a, ea);
    position_at(&e, b, eb);
    position_at(&q, a, qa);
    position_at(&q, b, qb);

    /* calcTimeInterval.  Relative position query - entry along the span,
     * with s in [0,1] the fraction of the span elapsed:
     *   r(s) = r0 + w s,   r0 = qa - ea,   w = (qb - eb) - (qa - ea).
     * Squared distance minus d^2 is the degree-two polynomial
     *   f(s) = A s^2 + B s + C,  A = w.w,  B = 2 r0.w,  C = r0.r0 - d^2. */
    double r0[3], w[3];
    for (int k = 0; k < 3; k++) {
        r0[k] = qa[k] - ea[k];
        w[k] = (qb[k] - eb[k]) - r0[k];
        if (ORACLE_MUTANT == 1) w[k] = 0.0;
    }
    double A = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double r0w = r0[0] * w[0] + r0[1] * w[1] + r0[2] * w[2];
    double B = 2.0 * r0w;
    if (ORACLE_MUTANT == 2) B = -B;
    double C = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2] - d * d;

    /* Closest approach inside the span: the vertex of f clamped to [0,1]. */
    double sstar = 0.0;
    if (A > 0.0) {
        sstar = -r0w / A;
        if (sstar < 0.0) sstar = 0.0;
        if (sstar > 1.0) sstar = 1.0;
    }
    double rc[3];
    for (int k = 0; k < 3; k++)
        rc[k] = r0[k] + w[k] * sstar;
    double dm = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
    if (dmin) *dmin = dm;
    if (ORACLE_MUTANT == 5 ? !(dm < d) : !(dm <= d))
        return 0;

    /* Non-empty: the roots of f, clipped to [0,1]. */
    double slo, shi;
    if (A == 0.0) {
        /* Constant separation (parallel motion): the whole span. */
        slo = 0.0;
        shi = 1.0;
    } else {
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double qq = -0.5 * (B + (B >= 0.0 ? sq : -sq));
        double r1 = qq / A;
        double r2 = (qq != 0.0) ? C / qq : r1;
        if (ORACLE_MUTANT == 6 && C != 0.0) r2 = qq / C;
        double lo = r1 < r2 ? r1 : r2;
        double hi = r1 < r2 ? r2 : r1;
        slo = lo > 0.0 ? lo : 0.0;
        shi = hi < 1.0 ? hi : 1.0;
        if (slo > shi) { /* tangent contact lost to rounding */
            slo = sstar;
            shi = sstar;
        }
    }
    double L = b - a;
    *t_enter = (slo == 0.0) ? a : (slo == 1.0 ? b : a + slo * L);
    *t_exit = (shi == 1.0) ? b : (shi == 0.0 ? a : a + shi * L);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Result collection.                                                        */
typedef struct {
    int64_t *qi, *ei;
    double *tin, *tout, *dmin;
    int64_t count, cap;
} obuf;

static int obuf_push(obuf *b, int64_t qi, int64_t ei, double tin, double tout, double dm)
{
    if (b->count == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 1024;
        int64_t *nqi = realloc(b->qi, nc * sizeof(int64_t));
        if (!nqi) return -1;
        b->qi = nqi;
        int64_t *nei = realloc(b->ei, nc * sizeof(int64_t));
        if (!nei) return -1;
        b->ei = nei;
        double *a1 = realloc(b->tin, nc * sizeof(double));
        if (!a1) return -1;
        b->tin = a1;
        double *a2 = realloc(b->tout, nc * sizeof(double));
        if (!a2) return -1;
        b->tout = a2;
        double *a3 = realloc(b->dmin, nc * sizeof(double));
        if (!a3) return -1;
        b->dmin = a3;
        b->cap = nc;
    }
    b->qi[b->count] = qi;
    b->ei[b->count] = ei;
    b->tin[b->count] = tin;
    b->tout[b->count] = tout;
    b->dmin[b->count] = dm;
    b->count++;
    return 0;
}

static void obuf_free(obuf *b)
{
    free(b->qi); free(b->ei); free(b->tin); free(b->tout); free(b->dmin);
    memset(b, 0, sizeof *b);
}

/* Opaque result handle returned to the caller. */
typedef struct {
    obuf all;
    int64_t overlap_pairs;  /* pairs with a common span of positive length */
    int64_t visited_pairs;  /* pairs the driver looked at */
} oracle_result;

int64_t oracle_result_count(const oracle_result *r) { return r ? r->all.count : -1; }
int64_t oracle_result_overlap_pairs(const oracle_result *r) { return r ? r->overlap_pairs : -1; }
int64_t oracle_result_visited_pairs(const oracle_result *r) { return r ? r->visited_pairs : -1; }

void oracle_result_copy(const oracle_result *r, int64_t *qi, int64_t *ei, double *tin,
                        double *tout, double *dmin)
{
    int64_t n = r->all.count;
    if (n == 0) return;
    memcpy(qi, r->all.qi, n * sizeof(int64_t));
    memcpy(ei, r->all.ei, n * sizeof(int64_t));
    memcpy(tin, r->all.tin, n * sizeof(double));
    memcpy(tout, r->all.tout, n * sizeof(double));
    memcpy(dmin, r->all.dmin, n * sizeof(double));
}

void oracle_result_free(oracle_result *r)
{
    if (!r) return;
    obuf_free(&r->all);
    free(r);
}

static int merge_into(oracle_result *r, obuf *parts, int nparts)
{
    int64_t total = 0;
    for (int i = 0; i < nparts; i++) total += parts[i].count;
    obuf *o = &r->all;
    for (int i = 0; i < nparts; i++)
        for (int64_t j = 0; j < parts[i].count; j++)
            if (obuf_push(o, parts[i].qi[j], parts[i].ei[j], parts[i].tin[j], parts[i].tout[j],
                          parts[i].dmin[j]))
                return -1;
    (void)total;
    return 0;
}

static int max_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    return nthreads < 1 ? 1 : nthreads;
}

/* Every query segment against every entry segment.  Entry and query arrays are
 * the eight columns (x_start, y_start, z_start, t_start, x_end, y_end, z_end,
 * t_end), each n (resp. nq) long.  Results are indices into the inputs. */
oracle_result *oracle_search_bruteforce(const double *const *ent, int64_t n, const double *const *qry,
                                        int64_t nq, double d, double wt0, double wt1, int nthreads)
{
    nthreads = max_threads(nthreads);
    oracle_result *r = calloc(1, sizeof *r);
    obuf *parts = calloc(nthreads, sizeof(obuf));
    int64_t *ov = calloc(nthreads, sizeof(int64_t));
    if (!r || !parts || !ov) { free(r); free(parts); free(ov); return NULL; }
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t qi = 0; qi < nq; qi++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        oseg q = load_seg(qry, qi);
        for (int64_t ei = 0; ei < n; ei++) {
            oseg e = load_seg(ent, ei);
            double tin, tout, dm;
            int hit = oracle_pair((const double *)&e, (const double *)&q, d, wt0, wt1, &tin, &tout, &dm);
            if (hit >= 0) ov[tid]++;
            if (hit == 1 && obuf_push(&parts[tid], qi, ei, tin, tout, dm)) failed = 1;
        }
    }
    for (int i = 0; i < nthreads; i++) r->overlap_pairs += ov[i];
    r->visited_pairs = n * nq;
    if (!failed) failed = merge_into(r, parts, nthreads);
    for (int i = 0; i < nthreads; i++) obuf_free(&parts[i]);
    free(parts);
    free(ov);
    if (failed) { oracle_result_free(r); return NULL; }
    return r;
}

/* Sort helper: entry order by (t_start, input index). */
static const double *g_sort_ts;
static int cmp_ts(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ta = g_sort_ts[a], tb = g_sort_ts[b];
    if (ta < tb) return -1;
    if (ta > tb) return 1;
    return (a > b) - (a < b);
}

/* Pair filter of the self-join (query (ii) of Sec. 2.1: every trajectory
 * against all other trajectories): a pair is reported only if its two
 * segments belong to different trajectories and, so that each unordered pair
 * appears once, the entry's id is larger than the query's.  NULL: no filter. */
typedef struct {
    const int64_t *etraj, *eseg, *qtraj, *qseg;
} pair_filter;

static int pair_allowed(const pair_filter *f, int64_t qi, int64_t ei)
{
    if (!f) return 1;
    if (ORACLE_MUTANT == 9) return f->eseg[ei] > f->qseg[qi];          /* same trajectory kept */
    if (ORACLE_MUTANT == 10) return f->etraj[ei] != f->qtraj[qi];      /* both orders kept */
    return f->etraj[ei] != f->qtraj[qi] && f->eseg[ei] > f->qseg[qi];
}

/* Same result as oracle_search_bruteforce, visiting fewer pairs: entries are
 * sorted by t_start; an entry can share a span of positive length with query
 * segment q only if q.t_start - maxdur < e.t_start < q.t_end, where maxdur is
 * the longest entry duration.  The temporal-overlap count covers every pair,
 * filtered or not. */
static oracle_result *sweep(const double *const *ent, int64_t n, const double *const *qry, int64_t nq, double d,
                            double wt0, double wt1, int nthreads, const pair_filter *filt, const double *dv,
                            const double *w0v, const double *w1v)
{
    nthreads = max_threads(nthreads);
    oracle_result *r = calloc(1, sizeof *r);
    int64_t *order = malloc((n > 0 ? n : 1) * sizeof(int64_t));
    double *sts = malloc((n > 0 ? n : 1) * sizeof(double));
    obuf *parts = calloc(nthreads, sizeof(obuf));
    int64_t *ov = calloc(nthreads, sizeof(int64_t));
    int64_t *vis = calloc(nthreads, sizeof(int64_t));
    if (!r || !order || !sts || !parts || !ov || !vis) {
        free(r); free(order); free(sts); free(parts); free(ov); free(vis);
        return NULL;
    }
    double maxdur = 0.0;
    for (int64_t i = 0; i < n; i++) {
        order[i] = i;
        double du = ent[7][i] - ent[3][i];
        if (du > maxdur) maxdur = du;
    }
    g_sort_ts = ent[3];
    qsort(order, n, sizeof(int64_t), cmp_ts);
    for (int64_t i = 0; i < n; i++) sts[i] = ent[3][order[i]];

    int failed = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t qi = 0; qi < nq; qi++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        oseg q = load_seg(qry, qi);
        /* this query segment's threshold and window (its own, when given) */
        const double dq = dv ? dv[qi] : d;
        const double w0 = w0v ? w0v[qi] : wt0;
        const double w1 = w1v ? w1v[qi] : wt1;
        double lo_t = ORACLE_MUTANT == 11 ? q.t0 : q.t0 - maxdur, hi_t = q.t1;
        /* first sorted position with t_start > lo_t */
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (sts[mid] > lo_t) hi = mid; else lo = mid + 1;
        }
        int64_t first = lo;
        /* first sorted position with t_start >= hi_t */
        lo = first; hi = n;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (sts[mid] >= hi_t) hi = mid; else lo = mid + 1;
        }
        int64_t last = lo;
        vis[tid] += last - first;
        for (int64_t k = first; k < last; k++) {
            int64_t ei = order[k];
            oseg e = load_seg(ent, ei);
            double tin, tout, dm;
            int hit = oracle_pair((const double *)&e, (const double *)&q, dq, w0, w1, &tin, &tout, &dm);
            if (hit >= 0) ov[tid]++;
            if (hit == 1 && pair_allowed(filt, qi, ei) && obuf_push(&parts[tid], qi, ei, tin, tout, dm)) failed = 1;
        }
    }
    for (int i = 0; i < nthreads; i++) {
        r->overlap_pairs += ov[i];
        r->visited_pairs += vis[i];
    }
    if (!failed) failed = merge_into(r, parts, nthreads);
    for (int i = 0; i < nthreads; i++) obuf_free(&parts[i]);
    free(parts); free(ov); free(vis); free(order); free(sts);
    if (failed) { oracle_result_free(r); return NULL; }
    return r;
}

oracle_result *oracle_search_sweep(const double *const *ent, int64_t n, const double *const *qry,
                                   int64_t nq, double d, double wt0, double wt1, int nthreads)
{
    return sweep(ent, n, qry, nq, d, wt0, wt1, nthreads, NULL, NULL, NULL, NULL);
}

/* The time sweep with a threshold and a window per query segment: query
 * segment i is searched with d[i] over [t0[i], t1[i]] (a query trajectory's
 * own d and window, Sec. 3, given to each of its segments), so that query
 * trajectories with different parameters are searched in one call. */
oracle_result *oracle_search_sweep_per_query(const double *const *ent, int64_t n, const double *const *qry,
                                             int64_t nq, const double *d, const double *wt0, const double *wt1,
                                             int nthreads)
{
    return sweep(ent, n, qry, nq, 0.0, 0.0, 0.0, nthreads, NULL, d, wt0, wt1);
}

/* Self-join (query (ii) of Sec. 2.1 with the query set equal to the
 * database): every segment against every segment of another trajectory,
 * each unordered pair once (reported with the smaller id as the query).
 * traj and seg are the n trajectory and segment ids; results are indices. */
oracle_result *oracle_self_join(const double *const *ent, int64_t n, const int64_t *traj, const int64_t *seg,
                                double d, double wt0, double wt1, int nthreads)
{
    const pair_filter f = {traj, seg, traj, seg};
    return sweep(ent, n, ent, n, d, wt0, wt1, nthreads, &f, NULL, NULL, NULL);
}

/* Number of OpenMP threads a search with nthreads<=0 would use. */
int oracle_default_threads(void) { return max_threads(0); }

/* ------------------------------------------------------------------------ */
/* Temporal-bin index of Sec. 4 (Fig. 1).                                    */
/*
 * Entries are sorted by non-decreasing t_start (ties by input index); the
 * extent [tmin, tmax] is split into m bins of width b = (tmax - tmin)/m; an
 * entry goes to bin floor((t_start - tmin)/b), the last bin also taking
 * t_start == tmax.  Per bin:
 *   bin_start      = smallest t_start in the bin (the value Fig. 1 prints)
 *   bin_end        = largest t_end in the bin
 *   bin_first/last = sorted positions of its first and last entry
 * Empty bins get first = last = -1 and start = end = NaN.
 * order[] receives the sorted order (input indices).  Returns b.
 */
double oracle_bin_table(const double *ts, const double *te, int64_t n, int64_t m, int64_t *order,
                        double *bin_start, double *bin_end, int64_t *bin_first, int64_t *bin_last)
{
    double tmin = INFINITY, tmax = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        order[i] = i;
        if (ts[i] < tmin) tmin = ts[i];
        if (te[i] > tmax) tmax = te[i];
    }
    g_sort_ts = ts;
    qsort(order, n, sizeof(int64_t), cmp_ts);
    double b = (tmax - tmin) / (double)m;
    for (int64_t j = 0; j < m; j++) {
        bin_start[j] = NAN;
        bin_end[j] = NAN;
        bin_first[j] = -1;
        bin_last[j] = -1;
    }
    for (int64_t k = 0; k < n; k++) {
        int64_t i = order[k];
        int64_t j = (int64_t)floor((ts[i] - tmin) / b);
        if (ORACLE_MUTANT == 7) j = (int64_t)floor(ts[i] / b);
        if (j >= m) j = m - 1;
        if (j < 0) j = 0;
        if (bin_first[j] < 0) {
            bin_first[j] = k;
            bin_start[j] = ts[i];
            bin_end[j] = te[i];
        }
        bin_last[j] = k;
        if (te[i] > bin_end[j]) bin_end[j] = te[i];
    }
    return b;
}

/*
 * Interactions of a query batching over a bin table (Sec. 4, Fig. 2): a batch
 * with cnt query segments and temporal extent [bts, bte] is compared with
 * every entry of every bin whose temporal extent [start_j, end_j] meets
 * [bts, bte] (closed intervals); it costs cnt * (entries in those bins).
 * The bin extent's lower end is passed in (the paper gives two readings:
 * j*b in the text, the smallest t_start in the figure).
 */
int64_t oracle_batch_interactions(const double *bin_lo, const double *bin_end, const int64_t *bin_first,
                                  const int64_t *bin_last, int64_t m, const int64_t *cnt,
                                  const double *bts, const double *bte, int64_t nb)
{
    int64_t total = 0;
    for (int64_t k = 0; k < nb; k++) {
        int64_t entries = 0;
        for (int64_t j = 0; j < m; j++) {
            if (bin_first[j] < 0) continue;
            if (bin_lo[j] <= bte[k] && bin_end[j] >= bts[k])
                entries += bin_last[j] - bin_first[j] + 1;
        }
        total += cnt[k] * entries;
    }
    return total;
}
