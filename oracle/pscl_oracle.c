/*
 * pscl_oracle.c -- plain, slow CPU reference for the two-level sampling-based
 * clustering of "A parallel sampling based clustering" (Sastry & Netti, arXiv 1412.1947).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header, table or helper
 * with the CUDA library and never calls it.  Build with -O2 -ffp-contract=off (no
 * -ffast-math): every floating-point operation below is one IEEE double operation
 * rounded to nearest, in the order written.
 *
 * What it computes, step by step in the paper's order:
 *   1. feature scaling of every attribute (Algorithm 1, step 1), min-max to [0,1];
 *   2. the equal-sized subclustering peel (Algorithm 1, steps 2-5, looped over the
 *      points left out as §II describes): landmark L = per-attribute minimum of the
 *      remaining points, squared Euclidean distance of every remaining point to L, the
 *      N nearest form one subcluster, they are removed, repeat until none remain;
 *   3. Lloyd's k-means (§I) on every subcluster to get its local centers
 *      (Algorithm 1, step 4);
 *   4. the pooled local centers are clustered once more with Lloyd (§V) to get the
 *      final centers;
 *   5. the sum of squared errors of all scaled points against the final centers.
 * Step 2 can instead be the unequal-sized subclustering of Algorithm 2: m landmarks
 * spaced along the segment from the per-attribute minimum L to the per-attribute
 * maximum H, every point grouped with its nearest landmark.
 *
 * Readings where the paper is silent (each is a choice, stated once here):
 *   - scaling: x' = RN_storage( (double(x) - mn) * (1 / (mx - mn)) ), the reciprocal and
 *     the product in double, rounded once to the job's storage type (float32, or bfloat16
 *     kept in a float); a constant attribute scales to 0;
 *   - distance: squared Euclidean, summed over attributes j = 0..d-1 in ascending order;
 *   - peel ties: equal distances are taken in ascending point index;
 *   - the landmark is recomputed over the remaining points every round;
 *   - the last subcluster holds the n mod N points left (if N does not divide n);
 *   - Lloyd starts from k_eff = min(k, m) members drawn by a seeded partial
 *     Fisher-Yates shuffle (SplitMix64 stream keyed by seed, stage, subcluster), runs
 *     exactly T iterations, breaks assignment ties by the lower center index and keeps
 *     an empty cluster's previous center;
 *   - the pooled set is the unweighted list of local centers in (subcluster, center)
 *     order;
 *   - Algorithm 2 ("divide the line segment between H and L into the required number
 *     of points"): landmark i of m sits at the middle of the i-th of m equal pieces,
 *     l_i = float(L + ((i + 1/2) / m) * (H - L)) per attribute in double; a point joins
 *     the landmark at the smallest squared distance (same summation as the peel),
 *     the lower landmark index on ties; landmarks nobody joins form no subcluster, and
 *     the subclusters are numbered in landmark order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

/* ------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", */
/* OOPSLA 2014): state advances by the golden-ratio increment, output is the mix.      */
/* ------------------------------------------------------------------------------ */
uint64_t or_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream of one Lloyd initialisation: stage 0 = a subcluster's local Lloyd (segment =
 * subcluster number), stage 1 = the final Lloyd on the pooled centers (segment 0).
 * The key is the SplitMix64 output for state (stage << 32 | segment), xor-ed into the
 * user's seed. */
uint64_t or_init_state(uint64_t seed, uint32_t stage, uint32_t segment)
{
    uint64_t key = ((uint64_t)stage << 32) | (uint64_t)segment;
    return seed ^ or_splitmix64_next(&key);
}

/* The first k positions of a Fisher-Yates shuffle of 0..m-1: at step i (0 <= i < k)
 * position i is swapped with position i + (r mod (m - i)), r the next stream value. */
int or_init_indices(uint64_t seed, uint32_t stage, uint32_t segment, int64_t m, int32_t k,
                    int64_t *out)
{
    int64_t i, *a;
    uint64_t st;
    if (m < 1 || k < 1 || k > m) return OR_EINVAL;
    a = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!a) return OR_ENOMEM;
    for (i = 0; i < m; i++) a[i] = i;
    st = or_init_state(seed, stage, segment);
    for (i = 0; i < k; i++) {
        uint64_t r = or_splitmix64_next(&st);
        int64_t j = i + (int64_t)(r % (uint64_t)(m - i));
        int64_t t = a[i];
        a[i] = a[j];
        a[j] = t;
    }
    for (i = 0; i < k; i++) out[i] = a[i];
    free(a);
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Step 1: feature scaling (Algorithm 1 step 1; the paper leaves the method open and */
/* min-max to [0,1] is used).                                                          */
/* ------------------------------------------------------------------------------ */
/* v rounded to nearest (ties to even) with 8 significant bits and bfloat16's exponent
 * range (subnormal spacing 2^-133), directly from double. */
static float round_bf16(double v)
{
    int e;
    double m, r;
    if (v == 0.0 || !isfinite(v)) return (float)v;
    if (fabs(v) < ldexp(1.0, -126)) return (float)(nearbyint(ldexp(v, 133)) * ldexp(1.0, -133));
    m = frexp(v, &e);                         /* v = m 2^e, 0.5 <= |m| < 1 */
    r = nearbyint(ldexp(m, 8));               /* 8 significant bits, ties to even */
    return (float)ldexp(r, e - 8);
}

int or_scale_storage(const float *raw, int64_t n, int32_t d, float *out, double *mn, double *mx, int bf16)
{
    int64_t i;
    int32_t j;
    if (n < 1 || d < 1) return OR_EINVAL;
    for (j = 0; j < d; j++) {
        double lo = (double)raw[j], hi = (double)raw[j];
        for (i = 1; i < n; i++) {
            double v = (double)raw[i * d + j];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        mn[j] = lo;
        mx[j] = hi;
    }
    for (j = 0; j < d; j++) {
        double range = mx[j] - mn[j];
        double inv = range > 0.0 ? 1.0 / range : 0.0;
        for (i = 0; i < n; i++) {
            if (range > 0.0) {
                double t = (double)raw[i * d + j] - mn[j];
                out[i * d + j] = bf16 ? round_bf16(t * inv) : (float)(t * inv);
            } else {
                out[i * d + j] = 0.0f;
            }
        }
    }
    return OR_OK;
}

int or_scale(const float *raw, int64_t n, int32_t d, float *out, double *mn, double *mx)
{
    return or_scale_storage(raw, n, d, out, mn, mx, 0);
}

/* ------------------------------------------------------------------------------ */
/* Squared Euclidean distance between a stored point and a double vector, summed in  */
/* ascending attribute order, one rounding per operation.                            */
/* ------------------------------------------------------------------------------ */
static double sqdist(const float *x, const double *c, int32_t d)
{
    double s = 0.0;
    int32_t j;
    for (j = 0; j < d; j++) {
        double diff = (double)x[j] - c[j];
        double sq = diff * diff;
        s = s + sq;
    }
    return s;
}

/* ------------------------------------------------------------------------------ */
/* Step 2: equal-sized subclustering (Algorithm 1 steps 2, 3 and 5; §II's "redoing  */
/* this process from the left out points").                                          */
/* ------------------------------------------------------------------------------ */
typedef struct { double key; int64_t idx; } keyed;

static int cmp_keyed(const void *a, const void *b)
{
    const keyed *p = (const keyed *)a, *q = (const keyed *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    if (p->idx < q->idx) return -1;
    if (p->idx > q->idx) return 1;
    return 0;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t p = *(const int64_t *)a, q = *(const int64_t *)b;
    return (p > q) - (p < q);
}

/* x: n*d scaled points.  Outputs: perm[n] (the points of subcluster s are
 * perm[seg_off[s] .. seg_off[s+1]-1], in ascending index), seg_off[S+1], *n_seg = S,
 * landmarks[S*d] (optional, the L of every round). */
int or_peel(const float *x, int64_t n, int32_t d, int64_t N, int64_t *perm, int64_t *seg_off,
            int64_t *n_seg, float *landmarks)
{
    int64_t *rem, nr, pos = 0, S = 0, i;
    keyed *kd;
    double *L;
    int32_t j;
    if (n < 1 || d < 1 || N < 1) return OR_EINVAL;
    rem = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    kd = (keyed *)malloc((size_t)n * sizeof(keyed));
    L = (double *)malloc((size_t)d * sizeof(double));
    if (!rem || !kd || !L) { free(rem); free(kd); free(L); return OR_ENOMEM; }
    for (i = 0; i < n; i++) rem[i] = i;
    nr = n;
    while (nr > 0) {
        int64_t take;
        /* the landmark: lowest value of every attribute over the remaining points */
        for (j = 0; j < d; j++) {
            float lo = x[rem[0] * d + j];
            for (i = 1; i < nr; i++) {
                float v = x[rem[i] * d + j];
                if (v < lo) lo = v;
            }
            L[j] = (double)lo;
            if (landmarks) landmarks[S * d + j] = lo;
        }
        /* distance of every remaining point to L; order by (distance, index) */
        for (i = 0; i < nr; i++) {
            kd[i].key = sqdist(x + rem[i] * d, L, d);
            kd[i].idx = rem[i];
        }
        qsort(kd, (size_t)nr, sizeof(keyed), cmp_keyed);
        /* the N closest form subcluster S (in ascending index), the rest remain */
        take = nr < N ? nr : N;
        seg_off[S] = pos;
        for (i = 0; i < take; i++) perm[pos + i] = kd[i].idx;
        qsort(perm + pos, (size_t)take, sizeof(int64_t), cmp_i64);
        pos += take;
        S++;
        for (i = take; i < nr; i++) rem[i - take] = kd[i].idx;
        nr -= take;
        qsort(rem, (size_t)nr, sizeof(int64_t), cmp_i64);
    }
    seg_off[S] = n;
    *n_seg = S;
    free(rem);
    free(kd);
    free(L);
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Nearest and second-nearest center of every point (lowest index on ties).          */
/* ------------------------------------------------------------------------------ */
int or_assign(const float *pts, int64_t m, int32_t d, const double *c, int32_t k,
              int32_t *labels, double *best, double *second)
{
    int64_t p;
    int32_t j;
    if (m < 0 || d < 1 || k < 1) return OR_EINVAL;
    for (p = 0; p < m; p++) {
        double b = INFINITY, s = INFINITY;
        int32_t bj = 0;
        for (j = 0; j < k; j++) {
            double v = sqdist(pts + p * d, c + (int64_t)j * d, d);
            if (v < b) { s = b; b = v; bj = j; }
            else if (v < s) { s = v; }
        }
        labels[p] = bj;
        if (best) best[p] = b;
        if (second) second[p] = s;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Lloyd's algorithm (§I): T rounds of "assign every point to its nearest center,    */
/* move every center to the mean of its points".                                      */
/*                                                                                    */
/* centers: k*d, in = initial centers, out = centers after T iterations.             */
/* labels:  m, the assignment of the last iteration.                                  */
/* sse_hist: T (optional), SSE after each iteration's update.                         */
/* counts:  k (optional), cluster sizes of the last iteration.                        */
/* force:   optional T*m labels from another implementation.  Where this oracle's    */
/*          own choice is not unique within tie_tol (the other choice's distance is  */
/*          within tie_tol*max(1, best) of the best), the other choice is followed;  */
/*          any other disagreement is counted in *n_bad.  NULL = plain Lloyd.          */
/* weights: optional m non-negative point weights (or_lloyd_w): a center moves to    */
/*          the weighted mean sum(w x) / sum(w) of its points, and sse_hist holds     */
/*          sum(w * distance).  With integer weights this is Lloyd on the multiset    */
/*          that holds point p w_p times.  NULL = every weight 1.                     */
/* ------------------------------------------------------------------------------ */
int or_lloyd_w(const float *pts, int64_t m, int32_t d, int32_t k, int32_t T, double *centers,
               int32_t *labels, double *sse_hist, int64_t *counts, const int64_t *weights,
               const int32_t *force, double tie_tol, int64_t *n_forced, int64_t *n_bad)
{
    double *sum;
    int64_t *cnt, p, forced = 0, bad = 0;
    int32_t t, j, a;
    if (m < 1 || d < 1 || k < 1 || T < 0) return OR_EINVAL;
    sum = (double *)malloc((size_t)k * d * sizeof(double));
    cnt = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    if (!sum || !cnt) { free(sum); free(cnt); return OR_ENOMEM; }
    for (t = 0; t < T; t++) {
        /* assignment */
        for (p = 0; p < m; p++) {
            double b = INFINITY;
            int32_t bj = 0;
            for (j = 0; j < k; j++) {
                double v = sqdist(pts + p * d, centers + (int64_t)j * d, d);
                if (v < b) { b = v; bj = j; }
            }
            if (force) {
                int32_t f = force[(int64_t)t * m + p];
                if (f != bj) {
                    double lim = tie_tol * (b > 1.0 ? b : 1.0);
                    if (f >= 0 && f < k &&
                        sqdist(pts + p * d, centers + (int64_t)f * d, d) - b <= lim) {
                        bj = f;
                        forced++;
                    } else {
                        bad++;
                    }
                }
            }
            labels[p] = bj;
        }
        /* update: mean of the members; an empty cluster keeps its center */
        memset(sum, 0, (size_t)k * d * sizeof(double));
        memset(cnt, 0, (size_t)k * sizeof(int64_t));
        for (p = 0; p < m; p++) {
            int32_t l = labels[p];
            if (weights) {
                cnt[l] += weights[p];
                for (a = 0; a < d; a++)
                    sum[(int64_t)l * d + a] = sum[(int64_t)l * d + a] + (double)weights[p] * (double)pts[p * d + a];
            } else {
                cnt[l] += 1;
                for (a = 0; a < d; a++) sum[(int64_t)l * d + a] = sum[(int64_t)l * d + a] + (double)pts[p * d + a];
            }
        }
        for (j = 0; j < k; j++) {
            if (cnt[j] > 0) {
                for (a = 0; a < d; a++)
                    centers[(int64_t)j * d + a] = sum[(int64_t)j * d + a] / (double)cnt[j];
            }
        }
        if (sse_hist) {
            double s = 0.0;
            for (p = 0; p < m; p++) {
                double v = sqdist(pts + p * d, centers + (int64_t)labels[p] * d, d);
                s = s + (weights ? (double)weights[p] * v : v);
            }
            sse_hist[t] = s;
        }
    }
    if (counts) {
        memset(cnt, 0, (size_t)k * sizeof(int64_t));
        for (p = 0; p < m; p++) cnt[labels[p]] += 1;
        for (j = 0; j < k; j++) counts[j] = cnt[j];
    }
    if (n_forced) *n_forced += forced;
    if (n_bad) *n_bad += bad;
    free(sum);
    free(cnt);
    return OR_OK;
}

int or_lloyd(const float *pts, int64_t m, int32_t d, int32_t k, int32_t T, double *centers,
             int32_t *labels, double *sse_hist, int64_t *counts, const int32_t *force,
             double tie_tol, int64_t *n_forced, int64_t *n_bad)
{
    return or_lloyd_w(pts, m, d, k, T, centers, labels, sse_hist, counts, NULL, force, tie_tol, n_forced, n_bad);
}

/* Initial centers of one Lloyd run over m points: the k_eff = min(k, m) points picked
 * by the seeded shuffle, or (first_k != 0) simply the first k_eff points. */
static int init_centers(const float *pts, int64_t m, int32_t d, int32_t k_eff, uint64_t seed,
                        uint32_t stage, uint32_t segment, int first_k, double *c)
{
    int64_t *idx = (int64_t *)malloc((size_t)k_eff * sizeof(int64_t));
    int32_t j, a;
    int rc = OR_OK;
    if (!idx) return OR_ENOMEM;
    if (first_k) {
        for (j = 0; j < k_eff; j++) idx[j] = j;
    } else {
        rc = or_init_indices(seed, stage, segment, m, k_eff, idx);
    }
    if (rc == OR_OK)
        for (j = 0; j < k_eff; j++)
            for (a = 0; a < d; a++) c[(int64_t)j * d + a] = (double)pts[idx[j] * d + a];
    free(idx);
    return rc;
}

int or_lloyd_seeded(const float *pts, int64_t m, int32_t d, int32_t k, int32_t T, uint64_t seed,
                    uint32_t stage, uint32_t segment, int first_k, double *centers,
                    int32_t *labels, double *sse_hist, int64_t *counts)
{
    int32_t k_eff = (int64_t)k < m ? k : (int32_t)m;
    int rc = init_centers(pts, m, d, k_eff, seed, stage, segment, first_k, centers);
    if (rc != OR_OK) return rc;
    return or_lloyd(pts, m, d, k_eff, T, centers, labels, sse_hist, counts, NULL, 0.0, NULL, NULL);
}

/* ------------------------------------------------------------------------------ */
/* Step 2 alternative: unequal-sized subclustering (Algorithm 2).                    */
/* x: n*d scaled points, m landmarks.  Outputs as or_peel (groups with no point are   */
/* skipped, so *n_seg <= m); landmarks[m*d] (optional); group[n] (optional): the      */
/* landmark index of every point.                                                     */
/* ------------------------------------------------------------------------------ */
int or_group_unequal(const float *x, int64_t n, int32_t d, int32_t m, int64_t *perm, int64_t *seg_off,
                     int64_t *n_seg, float *landmarks, int32_t *group)
{
    double *lm, *lo, *hi;
    int64_t *cnt, *next, i;
    int32_t *g, j, a;
    int64_t S = 0;
    if (n < 1 || d < 1 || m < 1) return OR_EINVAL;
    lm = (double *)malloc((size_t)m * d * sizeof(double));
    lo = (double *)malloc((size_t)d * sizeof(double));
    hi = (double *)malloc((size_t)d * sizeof(double));
    cnt = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    next = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    g = group ? group : (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!lm || !lo || !hi || !cnt || !next || !g) {
        free(lm); free(lo); free(hi); free(cnt); free(next);
        if (!group) free(g);
        return OR_ENOMEM;
    }
    /* L and H: the lowest and highest value of every attribute */
    for (a = 0; a < d; a++) {
        lo[a] = (double)x[a];
        hi[a] = (double)x[a];
    }
    for (i = 1; i < n; i++)
        for (a = 0; a < d; a++) {
            double v = (double)x[i * d + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    /* the landmarks: middles of m equal pieces of the segment from L to H, stored as
     * float like the points */
    for (j = 0; j < m; j++) {
        double t = ((double)j + 0.5) / (double)m;
        for (a = 0; a < d; a++) {
            float v = (float)(lo[a] + t * (hi[a] - lo[a]));
            lm[(int64_t)j * d + a] = (double)v;
            if (landmarks) landmarks[(int64_t)j * d + a] = v;
        }
    }
    /* every point joins its nearest landmark (lower index on ties) */
    for (i = 0; i < n; i++) {
        double best = INFINITY;
        int32_t bj = 0;
        for (j = 0; j < m; j++) {
            double v = sqdist(x + i * d, lm + (int64_t)j * d, d);
            if (v < best) { best = v; bj = j; }
        }
        g[i] = bj;
        cnt[bj] += 1;
    }
    /* subclusters in landmark order, points in ascending index inside each */
    seg_off[0] = 0;
    for (j = 0; j < m; j++) {
        if (cnt[j] == 0) { next[j] = -1; continue; }
        next[j] = seg_off[S];
        seg_off[S + 1] = seg_off[S] + cnt[j];
        S++;
    }
    for (i = 0; i < n; i++) perm[next[g[i]]++] = i;
    *n_seg = S;
    free(lm); free(lo); free(hi); free(cnt); free(next);
    if (!group) free(g);
    return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* The whole method.                                                                   */
/* ------------------------------------------------------------------------------ */
typedef struct {
    /* inputs */
    const float *raw;
    int64_t n;
    int64_t N;
    int32_t d;
    int32_t local_k;
    int32_t final_k;
    int32_t iters;
    uint64_t seed;
    int32_t first_k;          /* 1: every Lloyd starts from its first k_eff points */
    int32_t n_threads;        /* threads over subclusters (0 = library default)    */
    int32_t select_peel;      /* 1: or_peel_select instead of or_peel (same result) */
    int32_t unequal_m;        /* > 0: Algorithm 2 with this many landmarks instead of the peel */
    int32_t storage_bf16;     /* 1: scaled values rounded to bfloat16 (raw: bfloat16 values) */
    int32_t pool_weighted;    /* 1: the pooled Lloyd weighs every local center by its cluster's
                                 size in the last local iteration (the abstract clusters the
                                 subclusters' means; the sizes make that the weighted means) */
    const int32_t *force_local; /* optional iters*n trace, subcluster-packed order */
    const int32_t *force_final; /* optional iters*P trace                          */
    double tie_tol;
    /* outputs, caller-allocated (S = ceil(n/N), P = sum of min(local_k, |s|)) */
    float *scaled;            /* n*d */
    int64_t *perm;            /* n   */
    int64_t *seg_off;         /* S+1 */
    float *landmarks;         /* S*d, or unequal_m*d (optional) */
    double *local_centers;    /* P*d */
    int32_t *local_k_eff;     /* S */
    int32_t *local_labels;    /* n, subcluster-packed order (optional) */
    double *local_sse;        /* S*iters (optional) */
    double *final_centers;    /* final_k*d */
    double *final_sse_hist;   /* iters (optional) */
    int32_t *final_labels_pooled; /* P (optional) */
    int32_t *labels;          /* n (optional): nearest final center of every point */
    double *best;             /* n (optional) */
    double *second;           /* n (optional) */
    double sse;
    int64_t n_seg;
    int64_t n_pooled;
    int64_t n_forced;
    int64_t n_bad;
} or_two_level_args;

int or_peel_select(const float *x, int64_t n, int32_t d, int64_t N, int64_t *perm, int64_t *seg_off,
                   int64_t *n_seg, float *landmarks);

int or_two_level(or_two_level_args *A)
{
    int64_t n = A->n, S, P = 0, s, i;
    int32_t d = A->d, T = A->iters;
    double *mn, *mx;
    float *packed;
    int64_t *cen_off;
    int64_t *wts = NULL;      /* pooled weights (pool_weighted) */
    int rc;
    if (n < 1 || d < 1 || A->N < 1 || A->local_k < 1 || A->final_k < 1 || T < 0) return OR_EINVAL;
    mn = (double *)malloc((size_t)d * sizeof(double));
    mx = (double *)malloc((size_t)d * sizeof(double));
    packed = (float *)malloc((size_t)n * d * sizeof(float));
    cen_off = (int64_t *)malloc((size_t)(n / A->N + 2 + (A->unequal_m > 0 ? A->unequal_m : 0)) * sizeof(int64_t));
    if (!mn || !mx || !packed || !cen_off) { rc = OR_ENOMEM; goto done; }

    rc = or_scale_storage(A->raw, n, d, A->scaled, mn, mx, A->storage_bf16);
    if (rc) goto done;
    if (A->unequal_m > 0)
        rc = or_group_unequal(A->scaled, n, d, A->unequal_m, A->perm, A->seg_off, &S, A->landmarks, NULL);
    else if (A->select_peel)
        rc = or_peel_select(A->scaled, n, d, A->N, A->perm, A->seg_off, &S, A->landmarks);
    else
        rc = or_peel(A->scaled, n, d, A->N, A->perm, A->seg_off, &S, A->landmarks);
    if (rc) goto done;
    A->n_seg = S;
    /* subcluster-packed copy of the points ("flattening while subgrouping", §V) */
    for (i = 0; i < n; i++) memcpy(packed + i * d, A->scaled + A->perm[i] * d, (size_t)d * sizeof(float));
    for (s = 0; s < S; s++) {
        int64_t m = A->seg_off[s + 1] - A->seg_off[s];
        int32_t ke = (int64_t)A->local_k < m ? A->local_k : (int32_t)m;
        A->local_k_eff[s] = ke;
        cen_off[s] = P;
        P += ke;
    }
    A->n_pooled = P;
    if (A->final_k > P) { rc = OR_EINVAL; goto done; }
    /* pooled weights: the local cluster sizes (no iteration, no sizes: every weight 1) */
    if (A->pool_weighted && T > 0) {
        wts = (int64_t *)malloc((size_t)P * sizeof(int64_t));
        if (!wts) { rc = OR_ENOMEM; goto done; }
    }

    /* Step 3: Lloyd on every subcluster (independent, so they may run concurrently). */
    {
        int64_t forced = 0, bad = 0;
        int err = 0;
#ifdef _OPENMP
        int nt = A->n_threads > 0 ? A->n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : forced, bad) reduction(| : err)
#endif
        for (s = 0; s < S; s++) {
            int64_t off = A->seg_off[s], m = A->seg_off[s + 1] - off, t;
            int32_t ke = A->local_k_eff[s];
            int32_t *lab = A->local_labels ? A->local_labels + off : (int32_t *)malloc((size_t)m * sizeof(int32_t));
            double *hist = A->local_sse ? A->local_sse + s * T : NULL;
            int32_t *frc = NULL;
            int r2;
            if (!lab) { err |= 1; continue; }
            r2 = init_centers(packed + off * d, m, d, ke, A->seed, 0u, (uint32_t)s, A->first_k,
                              A->local_centers + cen_off[s] * d);
            if (r2 == OR_OK && A->force_local) {
                /* this subcluster's slice of the other implementation's trace */
                frc = (int32_t *)malloc((size_t)T * m * sizeof(int32_t));
                if (!frc) r2 = OR_ENOMEM;
                else for (t = 0; t < T; t++) memcpy(frc + t * m, A->force_local + t * n + off, (size_t)m * sizeof(int32_t));
            }
            if (r2 == OR_OK)
                r2 = or_lloyd(packed + off * d, m, d, ke, T, A->local_centers + cen_off[s] * d, lab,
                              hist, wts ? wts + cen_off[s] : NULL, frc, A->tie_tol, &forced, &bad);
            if (r2 != OR_OK) err |= 1;
            free(frc);
            if (!A->local_labels) free(lab);
        }
        A->n_forced = forced;
        A->n_bad = bad;
        if (err) { rc = OR_ENOMEM; goto done; }
    }

    /* Step 4: Lloyd on the pooled local centers (§V). */
    {
        float *pool = (float *)malloc((size_t)P * d * sizeof(float));
        int32_t *lab = A->final_labels_pooled ? A->final_labels_pooled : (int32_t *)malloc((size_t)P * sizeof(int32_t));
        int64_t forced = 0, bad = 0;
        if (!pool || !lab) { free(pool); if (!A->final_labels_pooled) free(lab); rc = OR_ENOMEM; goto done; }
        /* the pooled points are the local centers, stored like the data (float) */
        for (i = 0; i < P * d; i++) pool[i] = (float)A->local_centers[i];
        rc = init_centers(pool, P, d, A->final_k, A->seed, 1u, 0u, A->first_k, A->final_centers);
        if (rc == OR_OK)
            rc = or_lloyd_w(pool, P, d, A->final_k, T, A->final_centers, lab, A->final_sse_hist, NULL, wts,
                            A->force_final, A->tie_tol, &forced, &bad);
        A->n_forced += forced;
        A->n_bad += bad;
        free(pool);
        if (!A->final_labels_pooled) free(lab);
        if (rc) goto done;
    }

    /* Step 5: SSE of every scaled point against the final centers. */
    {
        double sse = 0.0;
        for (i = 0; i < n; i++) {
            double b = INFINITY, s2 = INFINITY;
            int32_t bj = 0, j;
            for (j = 0; j < A->final_k; j++) {
                double v = sqdist(A->scaled + i * d, A->final_centers + (int64_t)j * d, d);
                if (v < b) { s2 = b; b = v; bj = j; }
                else if (v < s2) { s2 = v; }
            }
            if (A->labels) A->labels[i] = bj;
            if (A->best) A->best[i] = b;
            if (A->second) A->second[i] = s2;
            sse = sse + b;
        }
        A->sse = sse;
    }
    rc = OR_OK;
done:
    free(mn);
    free(mx);
    free(packed);
    free(cen_off);
    free(wts);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* The same peel with a selection instead of a sort: per round, the N-th smallest     */
/* distance K is found by quickselect; the subcluster is every remaining point with   */
/* distance < K plus, in ascending index, as many with distance == K as are needed.   */
/* Identical output to or_peel (pinned by the tests), O(n_r) per round.               */
/* ------------------------------------------------------------------------------ */
static double kth_smallest(double *a, int64_t n, int64_t k)
{
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2, i = lo, j = hi;
        double x = a[lo], y = a[mid], z = a[hi], pivot, t;
        /* median of three */
        if ((x <= y && y <= z) || (z <= y && y <= x)) pivot = y;
        else if ((y <= x && x <= z) || (z <= x && x <= y)) pivot = x;
        else pivot = z;
        while (i <= j) {
            while (a[i] < pivot) i++;
            while (a[j] > pivot) j--;
            if (i <= j) { t = a[i]; a[i] = a[j]; a[j] = t; i++; j--; }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return a[k];
    }
    return a[k];
}

int or_peel_select(const float *x, int64_t n, int32_t d, int64_t N, int64_t *perm, int64_t *seg_off,
                   int64_t *n_seg, float *landmarks)
{
    int64_t *rem, nr, pos = 0, S = 0, i;
    double *delta, *tmp, *L;
    int32_t j;
    if (n < 1 || d < 1 || N < 1) return OR_EINVAL;
    rem = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    delta = (double *)malloc((size_t)n * sizeof(double));
    tmp = (double *)malloc((size_t)n * sizeof(double));
    L = (double *)malloc((size_t)d * sizeof(double));
    if (!rem || !delta || !tmp || !L) { free(rem); free(delta); free(tmp); free(L); return OR_ENOMEM; }
    for (i = 0; i < n; i++) rem[i] = i;
    nr = n;
    while (nr > 0) {
        int64_t kept = 0, take, need;
        double K;
        for (j = 0; j < d; j++) {
            float lo = x[rem[0] * d + j];
            for (i = 1; i < nr; i++) {
                float v = x[rem[i] * d + j];
                if (v < lo) lo = v;
            }
            L[j] = (double)lo;
            if (landmarks) landmarks[S * d + j] = lo;
        }
        for (i = 0; i < nr; i++) delta[i] = sqdist(x + rem[i] * d, L, d);
        seg_off[S] = pos;
        if (nr <= N) {
            for (i = 0; i < nr; i++) perm[pos + i] = rem[i];
            pos += nr;
            S++;
            break;
        }
        memcpy(tmp, delta, (size_t)nr * sizeof(double));
        K = kth_smallest(tmp, nr, N - 1);
        need = N;
        for (i = 0; i < nr; i++) need -= delta[i] < K;
        take = 0;
        for (i = 0; i < nr; i++) {         /* rem is in ascending index order */
            int sel = delta[i] < K || (delta[i] == K && need > 0);
            if (delta[i] == K && sel) need--;
            if (sel) perm[pos + take++] = rem[i];
            else rem[kept++] = rem[i];
        }
        pos += take;
        S++;
        nr = kept;
    }
    seg_off[S] = n;
    *n_seg = S;
    free(rem);
    free(delta);
    free(tmp);
    free(L);
    return OR_OK;
}
