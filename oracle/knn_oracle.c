/*
 * knn_oracle.c -- CPU oracle for the exact K-nearest-neighbour self-join.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library; the GPU library never does and
 * shares no code with it.
 *
 * What is computed (paper Sec. 2.1, problem statement): for every point p_i
 * of the data set D, its K nearest neighbours under the Euclidean distance,
 * the point itself excluded.  The paper fixes neither precision nor the order
 * of equal distances; this oracle makes both total:
 *
 *   D(i,j) = fl64(...fl64(fl64(t_0) + fl64(t_1)) + ... + fl64(t_{d-1})),
 *   t_k    = fl64(fl64((double)x_ik - (double)x_jk)^2),
 *
 * summed left to right with no fused multiply-add (build with
 * -ffp-contract=off), neighbours ranked by (D(i,j), j) ascending, and the
 * reported distance is the correctly rounded sqrt(D(i,j)).  Self-exclusion
 * is by index: another point with the same coordinates is a neighbour at
 * distance 0.
 *
 * Functions:
 *   oracle_bf       brute force over all pairs (the definition written out).
 *   oracle_bf_rows  the same for a chosen subset of query rows.
 *   oracle_bf_rs    brute force of the R x S join: for each query point of
 *                   a set R, the K nearest points of a data set S under the
 *                   same order, nothing excluded (the self-join applied to a
 *                   query set apart from the data, as Sec. 2.1 notes).
 *   oracle_fp32_rows  for chosen query rows, the K nearest under the FP32
 *                   filter distance alone (see below): what ranking without
 *                   the FP64 re-score would return.
 *   oracle_grid     an exact grid join in the paper's manner (Sec. 3.1 grid of
 *                   non-empty cells, Sec. 4.4 epsilon selection, ring of 3^n
 *                   adjacent cells, failed queries retried with a wider
 *                   search); it also counts the candidate distance
 *                   evaluations of that schedule.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* ------------------------------------------------------------------ */
/* Canonical squared distance (problem statement, Sec. 2.1).           */
/* ------------------------------------------------------------------ */
static double canon_d2(const float *a, const float *b, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        double sq = t * t;
#ifdef ORACLE_MUTANT_DROP_LAST_TERM
        if (k == d - 1 && d > 1) break;
#endif
        s = s + sq;
    }
    return s;
}

/* (D, id) order; the oracle's tie-break. */
static inline int nb_less(double da, int32_t ia, double db, int32_t ib)
{
#ifdef ORACLE_MUTANT_TIE_DESC
    return da < db || (da == db && ia > ib);
#else
    return da < db || (da == db && ia < ib);
#endif
}

typedef struct { double d2; int32_t id; } nb_t;

/* Keep the K smallest (d2, id) in top[0..cnt) sorted ascending. */
static inline void topk_insert(nb_t *top, int *cnt, int K, double d2, int32_t id)
{
    if (*cnt == K && !nb_less(d2, id, top[K - 1].d2, top[K - 1].id))
        return;
    int pos = (*cnt < K) ? (*cnt)++ : K - 1;
    while (pos > 0 && nb_less(d2, id, top[pos - 1].d2, top[pos - 1].id)) {
        top[pos] = top[pos - 1];
        --pos;
    }
    top[pos].d2 = d2;
    top[pos].id = id;
}

static void write_row(const nb_t *top, int K, int32_t *ids, double *dist)
{
    for (int k = 0; k < K; ++k) {
        ids[k] = top[k].id;
        dist[k] = sqrt(top[k].d2);
    }
}

static int threads_or_default(int nthreads)
{
    return nthreads > 0 ? nthreads : omp_get_max_threads();
}

/* ------------------------------------------------------------------ */
/* Brute force.                                                        */
/* ------------------------------------------------------------------ */
static void bf_one(const float *pts, int64_t n, int d, int K, int64_t i,
                   nb_t *top, int32_t *ids, double *dist)
{
    int cnt = 0;
    const float *q = pts + i * d;
    for (int64_t j = 0; j < n; ++j) {
#ifndef ORACLE_MUTANT_KEEP_SELF
        if (j == i) continue;
#endif
        topk_insert(top, &cnt, K, canon_d2(q, pts + j * d, d), (int32_t)j);
    }
    write_row(top, K, ids, dist);
}

/* Returns 0 on success, -1 on invalid arguments. */
int oracle_bf(const float *pts, int64_t n, int d, int K,
              int32_t *ids, double *dist, int nthreads)
{
    if (!pts || !ids || !dist || n < 2 || d < 1 || K < 1 || K > n - 1)
        return -1;
    int nt = threads_or_default(nthreads);
    #pragma omp parallel num_threads(nt)
    {
        nb_t *top = (nb_t *)malloc(sizeof(nb_t) * (size_t)K);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i)
            bf_one(pts, n, d, K, i, top, ids + i * K, dist + i * K);
        free(top);
    }
    return 0;
}

int oracle_bf_rows(const float *pts, int64_t n, int d, int K,
                   const int64_t *rows, int64_t nrows,
                   int32_t *ids, double *dist, int nthreads)
{
    if (!pts || !rows || !ids || !dist || n < 2 || d < 1 || K < 1 || K > n - 1)
        return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) return -1;
    int nt = threads_or_default(nthreads);
    #pragma omp parallel num_threads(nt)
    {
        nb_t *top = (nb_t *)malloc(sizeof(nb_t) * (size_t)K);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r)
            bf_one(pts, n, d, K, rows[r], top, ids + r * K, dist + r * K);
        free(top);
    }
    return 0;
}

/* R x S: every pair (r, j), ranked by (D(r, j), j); no exclusion. */
int oracle_bf_rs(const float *qry, int64_t nq, const float *pts, int64_t n, int d, int K,
                 int32_t *ids, double *dist, int nthreads)
{
    if (!qry || !pts || !ids || !dist || nq < 1 || n < 1 || d < 1 || K < 1 || K > n)
        return -1;
    int nt = threads_or_default(nthreads);
    #pragma omp parallel num_threads(nt)
    {
        nb_t *top = (nb_t *)malloc(sizeof(nb_t) * (size_t)K);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nq; ++r) {
            int cnt = 0;
            const float *q = qry + r * d;
            for (int64_t j = 0; j < n; ++j)
                topk_insert(top, &cnt, K, canon_d2(q, pts + j * d, d), (int32_t)j);
            write_row(top, K, ids + r * K, dist + r * K);
        }
        free(top);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* FP32-only ranking (diagnostic).                                     */
/*                                                                      */
/* The GPU join filters candidates with a single-precision squared      */
/* distance and ranks the survivors in canonical FP64.  The filter's    */
/* value, written here independently: every difference                 */
/* t_k = fl32(x_ik - x_jk); for d < 4 one accumulator                   */
/* s = fma32(t_k, t_k, s) over k = 0..d-1 (one rounding per fused       */
/* step); for d >= 4 two accumulators, even k into e and odd k into o,  */
/* each fma32(t_k, t_k, .), then fl32(e + o).  oracle_fp32_rows ranks   */
/* all j != i by (that value, j) and keeps the K smallest.  Parity      */
/* unpinned against the paper (which fixes no precision); pinned in the */
/* tests by an exact-rational emulation of single-precision rounding.   */
/* ------------------------------------------------------------------ */
static float filter_d2_32(const float *a, const float *b, int d)
{
#ifdef ORACLE_MUTANT_FP32_ONE_CHAIN
    if (d < 9) {
#else
    if (d < 4) {
#endif
        float s = 0.0f;
        for (int k = 0; k < d; ++k) {
            float t = a[k] - b[k];
#ifdef ORACLE_MUTANT_FP32_UNFUSED
            float sq = t * t;
            s = s + sq;
#else
            s = fmaf(t, t, s);
#endif
        }
        return s;
    }
    float e = 0.0f, o = 0.0f;
    for (int k = 0; k < d; ++k) {
        float t = a[k] - b[k];
        if (k & 1)
            o = fmaf(t, t, o);
        else
            e = fmaf(t, t, e);
    }
    return e + o;
}

int oracle_fp32_rows(const float *pts, int64_t n, int d, int K,
                     const int64_t *rows, int64_t nrows, int32_t *ids, int nthreads)
{
    if (!pts || !rows || !ids || n < 2 || d < 1 || K < 1 || K > n - 1)
        return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) return -1;
    int nt = threads_or_default(nthreads);
    #pragma omp parallel num_threads(nt)
    {
        nb_t *top = (nb_t *)malloc(sizeof(nb_t) * (size_t)K);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nrows; ++r) {
            int cnt = 0;
            const int64_t i = rows[r];
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                /* a float widened to double keeps its value and order */
                topk_insert(top, &cnt, K, (double)filter_d2_32(pts + i * d, pts + j * d, d), (int32_t)j);
            }
            for (int k = 0; k < K; ++k) ids[r * K + k] = top[k].id;
        }
        free(top);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid join.                                                          */
/*                                                                      */
/* Search distance (Sec. 4.4): sample about 0.1% of D and take the mean */
/* distance between the sampled points (eps_mean); histogram the        */
/* distances from a fixed sample of points to every other point of D    */
/* into n_bins bins of width eps_mean / n_bins (distances >= eps_mean   */
/* not stored); eps_min is the middle of the first bin whose cumulative */
/* count, averaged over the sampled points, reaches K.                  */
/*                                                                      */
/* Index (Sec. 3.1): cells of side w; only non-empty cells are stored.  */
/* A query in cell c is compared with the points of the 3^n cells       */
/* c + {-1,0,1}^n.  Its K-th neighbour is certain when the K-th         */
/* distance is smaller than the distance from the query to the faces of */
/* that 3^n box (points outside the box are at least that far).  A     */
/* query that is not certain is retried on the grid of twice the cell   */
/* side (a wider ring of cells), until the box covers every non-empty   */
/* cell, at which point it is certain.                                  */
/* ------------------------------------------------------------------ */

#define GRID_NBINS 1024
#define GRID_HIST_SAMPLES 500

typedef struct {
    double eps_mean, eps_min, width;
    int64_t candidates;      /* distance evaluations, all passes */
    int passes;
    int64_t pass_queries[64];
    int64_t pass_candidates[64];
} oracle_grid_stats;

/* floor(x / w) exactly, for w with at most 20 significant bits and
 * |x / w| < 2^32: q * w is then exact in double, so the comparisons are. */
static int64_t exact_floor_div(float xf, double w)
{
    double x = (double)xf;
    double q = floor(x / w);
    int64_t c = (int64_t)q;
    while ((double)c * w > x) --c;
    while ((double)(c + 1) * w <= x) ++c;
    return c;
}

static int64_t floor_shift(int64_t c, int l)
{
    /* floor(c / 2^l) for any sign */
    return c >= 0 ? (c >> l) : -((-c + ((int64_t)1 << l) - 1) >> l);
}

static double round_to_20_bits(double w)
{
    int e;
    double m = frexp(w, &e);             /* w = m * 2^e, m in [0.5, 1) */
    m = nearbyint(ldexp(m, 20));         /* 20-bit integer mantissa */
    return ldexp(m, e - 20);
}

double oracle_select_epsilon(const float *pts, int64_t n, int d, int K,
                             double *eps_mean_out, int nthreads)
{
    int nt = threads_or_default(nthreads);
    /* eps_mean: mean pairwise distance among ~0.1% of D (>= 2, <= 2000). */
    int64_t sm = (int64_t)llround(0.001 * (double)n);
    if (sm < 2) sm = 2;
    if (sm > 2000) sm = 2000;
    if (sm > n) sm = n;
    double sum = 0.0;
    int64_t pairs = 0;
    #pragma omp parallel for num_threads(nt) reduction(+:sum, pairs) schedule(dynamic, 8)
    for (int64_t a = 0; a < sm; ++a) {
        int64_t ia = a * (n / sm);
        for (int64_t b = a + 1; b < sm; ++b) {
            int64_t ib = b * (n / sm);
            sum += sqrt(canon_d2(pts + ia * d, pts + ib * d, d));
            ++pairs;
        }
    }
    double eps_mean = pairs ? sum / (double)pairs : 0.0;
    if (eps_mean_out) *eps_mean_out = eps_mean;
    if (!(eps_mean > 0.0)) return 0.0;

    /* Histogram of distances from S sampled points to all of D. */
    int64_t S = n < GRID_HIST_SAMPLES ? n : GRID_HIST_SAMPLES;
    double bw = eps_mean / GRID_NBINS;
    int64_t hist[GRID_NBINS];
    memset(hist, 0, sizeof(hist));
    #pragma omp parallel num_threads(nt)
    {
        int64_t h[GRID_NBINS];
        memset(h, 0, sizeof(h));
        #pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < S; ++s) {
            int64_t is = s * (n / S);
            for (int64_t j = 0; j < n; ++j) {
                if (j == is) continue;
                double dist = sqrt(canon_d2(pts + is * d, pts + j * d, d));
                if (dist < eps_mean) {
#ifdef ORACLE_MUTANT_EPS_BIN_OFF_BY_ONE
                    int64_t b = (int64_t)(dist / bw) + 1;
#else
                    int64_t b = (int64_t)(dist / bw);
#endif
                    if (b >= GRID_NBINS) b = GRID_NBINS - 1;
                    h[b]++;
                }
            }
        }
        #pragma omp critical
        for (int b = 0; b < GRID_NBINS; ++b) hist[b] += h[b];
    }
    int64_t cum = 0;
    for (int b = 0; b < GRID_NBINS; ++b) {
        cum += hist[b];
        if ((double)cum / (double)S >= (double)K)
            return (b + 0.5) * bw;   /* middle of [b*bw, (b+1)*bw) */
    }
    return eps_mean;
}

/* Sorted list of points by (cell tuple at a level, id), with a hash map
 * from cell tuple to its run in that list. */
typedef struct {
    int d;
    int64_t n;
    const int64_t *cell;     /* n x d cell coordinates at this level */
    int64_t *order;          /* point ids sorted by (cell tuple, id) */
    int64_t ncells;
    int64_t *run_start, *run_len;  /* per unique cell */
    int64_t hsize;
    int64_t *hslot;          /* hash slot -> unique cell index, -1 empty */
} level_index;

static int cmp_cells(const int64_t *a, const int64_t *b, int d)
{
    for (int k = 0; k < d; ++k) {
        if (a[k] < b[k]) return -1;
        if (a[k] > b[k]) return 1;
    }
    return 0;
}

static int cmp_order(const void *pa, const void *pb, void *ctx)
{
    const level_index *L = (const level_index *)ctx;
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    int c = cmp_cells(L->cell + a * L->d, L->cell + b * L->d, L->d);
    if (c) return c;
    return a < b ? -1 : (a > b);
}

static uint64_t hash_cell(const int64_t *c, int d)
{
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int k = 0; k < d; ++k) {
        h ^= (uint64_t)c[k] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 31;
    }
    return h;
}

static void level_build(level_index *L, const int64_t *cell, int64_t n, int d)
{
    L->d = d;
    L->n = n;
    L->cell = cell;
    L->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) L->order[i] = i;
    qsort_r(L->order, (size_t)n, sizeof(int64_t), cmp_order, L);
    L->run_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    L->run_len = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t m = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (s == 0 || cmp_cells(cell + L->order[s] * d, cell + L->order[s - 1] * d, d)) {
            L->run_start[m] = s;
            L->run_len[m] = 0;
            ++m;
        }
        L->run_len[m - 1]++;
    }
    L->ncells = m;
    int64_t hs = 1;
    while (hs < 2 * m) hs <<= 1;
    L->hsize = hs;
    L->hslot = (int64_t *)malloc(sizeof(int64_t) * (size_t)hs);
    for (int64_t h = 0; h < hs; ++h) L->hslot[h] = -1;
    for (int64_t u = 0; u < m; ++u) {
        const int64_t *c = cell + L->order[L->run_start[u]] * d;
        uint64_t h = hash_cell(c, d) & (uint64_t)(hs - 1);
        while (L->hslot[h] >= 0) h = (h + 1) & (uint64_t)(hs - 1);
        L->hslot[h] = u;
    }
}

static int64_t level_find(const level_index *L, const int64_t *c)
{
    uint64_t h = hash_cell(c, L->d) & (uint64_t)(L->hsize - 1);
    for (;;) {
        int64_t u = L->hslot[h];
        if (u < 0) return -1;
        if (!cmp_cells(L->cell + L->order[L->run_start[u]] * L->d, c, L->d)) return u;
        h = (h + 1) & (uint64_t)(L->hsize - 1);
    }
}

static void level_free(level_index *L)
{
    free(L->order);
    free(L->run_start);
    free(L->run_len);
    free(L->hslot);
}

/* Grid join of the query rows `rows` (all rows when rows == NULL) against
 * all of D; row r of ids/dist belongs to query rows[r] (or r).
 * Returns 0 on success, -1 on invalid arguments. */
int oracle_grid_rows(const float *pts, int64_t n, int d, int K, double width_mult,
                     const int64_t *rows, int64_t nrows,
                     int32_t *ids, double *dist, oracle_grid_stats *st, int nthreads)
{
    if (!pts || !ids || !dist || n < 2 || d < 1 || d > 16 || K < 1 || K > n - 1)
        return -1;
    if (rows)
        for (int64_t r = 0; r < nrows; ++r)
            if (rows[r] < 0 || rows[r] >= n) return -1;
    int nt = threads_or_default(nthreads);
    oracle_grid_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));

    double eps_mean = 0.0;
    double eps_min = oracle_select_epsilon(pts, n, d, K, &eps_mean, nt);
    st->eps_mean = eps_mean;
    st->eps_min = eps_min;

    double maxabs = 0.0;
    for (int64_t i = 0; i < n * d; ++i) {
        double a = fabs((double)pts[i]);
        if (a > maxabs) maxabs = a;
    }
    /* width_mult > 0 scales eps_min; width_mult < 0 sets the cell side to
     * -width_mult directly (used by tests that need faces at known places). */
    double w = width_mult < 0.0 ? -width_mult
                                : eps_min * (width_mult > 0.0 ? width_mult : 1.0);
    double wfloor = ldexp(maxabs, -31);
    if (!(w > wfloor)) w = wfloor;
    if (!(w > 0.0)) w = 1.0;          /* every coordinate is 0 */
    w = round_to_20_bits(w);
    if (w < wfloor) w = round_to_20_bits(2.0 * wfloor);
    st->width = w;

    /* Level-0 cell coordinates. */
    int64_t *c0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n * d));
    #pragma omp parallel for num_threads(nt)
    for (int64_t i = 0; i < n * d; ++i)
        c0[i] = exact_floor_div(pts[i], w);

    int64_t *cl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n * d));
    int64_t cap = (rows && nrows > n) ? nrows : n;
    int64_t *active = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    char *fail = (char *)malloc((size_t)cap);
    /* active entries are output rows; the query of row a is rows[a] (or a) */
    int64_t nactive = rows ? nrows : n;
    for (int64_t i = 0; i < nactive; ++i) active[i] = i;

    int64_t noffs = 1;
    for (int k = 0; k < d; ++k) noffs *= 3;

    for (int lvl = 0; nactive > 0; ++lvl) {
        double wl = ldexp(w, lvl);
        int64_t cmin[16], cmax[16];
        for (int k = 0; k < d; ++k) { cmin[k] = INT64_MAX; cmax[k] = INT64_MIN; }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < d; ++k) {
                int64_t c = floor_shift(c0[i * d + k], lvl);
                cl[i * d + k] = c;
                if (c < cmin[k]) cmin[k] = c;
                if (c > cmax[k]) cmax[k] = c;
            }
        level_index L;
        level_build(&L, cl, n, d);
        int64_t cand_total = 0;

        #pragma omp parallel num_threads(nt) reduction(+:cand_total)
        {
            nb_t *top = (nb_t *)malloc(sizeof(nb_t) * (size_t)K);
            int64_t nb[16];
            #pragma omp for schedule(dynamic, 256)
            for (int64_t a = 0; a < nactive; ++a) {
                int64_t row = active[a];
                int64_t i = rows ? rows[row] : row;
                const float *q = pts + i * d;
                const int64_t *cq = cl + i * d;
                int cnt = 0;
                for (int64_t o = 0; o < noffs; ++o) {
                    int64_t r = o;
                    int skip = 0;
                    for (int k = 0; k < d; ++k) {
                        nb[k] = cq[k] + (r % 3) - 1;
#ifdef ORACLE_MUTANT_NO_LOWER_NEIGHBOUR
                        if (nb[k] < cq[k]) skip = 1;
#endif
                        r /= 3;
                        if (nb[k] < cmin[k] || nb[k] > cmax[k]) skip = 1;
                    }
                    if (skip) continue;
                    int64_t u = level_find(&L, nb);
                    if (u < 0) continue;
                    for (int64_t s = L.run_start[u]; s < L.run_start[u] + L.run_len[u]; ++s) {
                        int64_t j = L.order[s];
#ifdef ORACLE_MUTANT_COUNT_SELF
                        if (j == i) { ++cand_total; continue; }
#else
                        if (j == i) continue;
#endif
                        ++cand_total;
                        topk_insert(top, &cnt, K, canon_d2(q, pts + j * d, d), (int32_t)j);
                    }
                }
                /* Certificate: distance to the faces of the scanned box.
                 * Faces are integer multiples of wl, exact in double; the
                 * rounded gap and square are within 2^-52 relative of the
                 * exact ones, and D of any point outside the box is at least
                 * (1 - 2^-50) times its exact squared distance, so the
                 * factor (1 - 2^-40) leaves a wide margin. */
                double R = INFINITY;
                for (int k = 0; k < d; ++k) {
                    if (cq[k] - 1 > cmin[k]) {
                        double g = (double)q[k] - (double)(cq[k] - 1) * wl;
                        if (g < R) R = g;
                    }
                    if (cq[k] + 1 < cmax[k]) {
                        double g = (double)(cq[k] + 2) * wl - (double)q[k];
                        if (g < R) R = g;
                    }
                }
                int ok = 0;
                if (cnt == K) {
#ifdef ORACLE_MUTANT_LOOSE_CERTIFICATE
                    ok = isinf(R) || top[K - 1].d2 <= R * R;
#else
                    ok = isinf(R) || top[K - 1].d2 < R * R * (1.0 - 0x1p-40);
#endif
                }
                fail[a] = (char)!ok;
                if (ok) write_row(top, K, ids + row * K, dist + row * K);
            }
            free(top);
        }
        level_free(&L);
        if (lvl < 64) {
            st->pass_queries[lvl] = nactive;
            st->pass_candidates[lvl] = cand_total;
        }
#ifdef ORACLE_MUTANT_COUNT_LAST_PASS
        st->candidates = cand_total;
#else
        st->candidates += cand_total;
#endif
        st->passes = lvl + 1;
        int64_t m = 0;
        for (int64_t a = 0; a < nactive; ++a)
            if (fail[a]) next[m++] = active[a];
        int64_t *tmp = active; active = next; next = tmp;
        nactive = m;
    }
    free(c0); free(cl); free(active); free(next); free(fail);
    return 0;
}

int oracle_grid(const float *pts, int64_t n, int d, int K, double width_mult,
                int32_t *ids, double *dist, oracle_grid_stats *st, int nthreads)
{
    return oracle_grid_rows(pts, n, d, K, width_mult, NULL, 0, ids, dist, st, nthreads);
}

/* Size of the stats struct, so the Python side can check its layout. */
int oracle_grid_stats_size(void) { return (int)sizeof(oracle_grid_stats); }
