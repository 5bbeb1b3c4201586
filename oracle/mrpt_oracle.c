/*
 * MRPT oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised CPU restatement of the multiple
 * random projection tree method with voting (Hyvonen et al., "Fast k-NN
 * search", arXiv:1509.06957).  It exists to check the CUDA library against.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the product library shares no code, header or table with it.
 *
 * Every function follows the paper's steps in the paper's order:
 *   - orc_random_matrix : Algorithm 1, inner two loops; Sec. II-B (sparse
 *                         vectors r_i ~ N(0,1) w.p. a, else 0); Sec. II-C (one
 *                         vector per tree level, R in R^{d x l}).
 *   - orc_random_matrix_fixed : the footnote of Sec. II-D (exactly ceil(a d)
 *                         nonzeros per vector), the ablation of Table III.
 *   - orc_project       : Algorithm 1 (P = XR) and Algorithm 3 (p = q^T R).
 *   - orc_grow_tree     : Algorithm 2 with the order-based median of Sec. II-A
 *                         (first ceil(c/2) points by projected order go left).
 *   - orc_route         : Algorithm 3 (p <= split goes left).
 *   - orc_votes         : Algorithm 4 and the voting definitions of Sec. III-A.
 *   - orc_knn           : knn(q, k, S) of Algorithm 4 -- brute force on S with
 *                         the Euclidean metric of Sec. I-A.
 *   - orc_query         : Algorithm 4 end to end for a batch of queries.
 *   - orc_brute_knn     : exact k-NN of Sec. I-A (ground truth for recall).
 *
 * Readings where the paper is silent (documented with the tests):
 *   - RNG: SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based
 *     generator; Bernoulli by u < a; normals by Box-Muller (1958) in double,
 *     rounded to float.  Counter of draw s in {0,1,2} for tree t, level j,
 *     dimension i is 3*((t*l + j)*d + i) + s.
 *   - Projection order: ascending dimension, each step one fused
 *     multiply-add (fmaf) starting from +0.0f.  Compile with
 *     -ffp-contract=off so that nothing else is fused.
 *   - Median ties: points ordered by (projection, id); split value is the
 *     projection of the ceil(c/2)-th point in that order.
 *   - Distances: double precision (mode 0) or sequential float (mode 1);
 *     k-NN order by (squared distance, id); output distance is the square
 *     root; rows with |S| < k are padded with id -1 and +inf.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG ---- */

/* The i-th output (i = 0, 1, ...) of SplitMix64 whose state starts at `seed`:
 * the state advances by the golden-ratio increment before every output, and
 * the output is the published mixing function of the new state. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform in [0, 1) from the top 53 bits. */
static double unit_open_right(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
/* Uniform in (0, 1] from the top 53 bits (safe for log). */
static double unit_open_left(uint64_t x) { return ((double)(x >> 11) + 1.0) * 0x1.0p-53; }

/*
 * Sparse random matrix for T trees of depth l (Algorithm 1, Sec. II-B/II-C).
 * Column c = t*l + j holds tree t's vector for level j.  Component i of that
 * vector is nonzero with probability `density` (the paper's a) and then
 * drawn from N(0,1).
 *
 * Output in compressed-column form: col_off[T*l+1], dim[nnz], val[nnz],
 * nonzeros of a column in ascending dimension.  If dim or val is NULL only
 * col_off is written.  Returns nnz.
 */
int64_t orc_random_matrix(int32_t T, int32_t l, int32_t d, float density, uint64_t seed,
                          int32_t *col_off, int32_t *dim, float *val)
{
    const double a = (double)density;
    const double two_pi = 2.0 * 3.14159265358979323846;
    int64_t nnz = 0;
    for (int32_t t = 0; t < T; ++t) {
        for (int32_t j = 0; j < l; ++j) {
            const int32_t c = t * l + j;
            col_off[c] = (int32_t)nnz;
            for (int32_t i = 0; i < d; ++i) {
                const uint64_t ctr = 3ULL * (((uint64_t)c * (uint64_t)d) + (uint64_t)i);
                const double z = unit_open_right(orc_splitmix64(seed, ctr));
                if (z < a) { /* Bernoulli(a) came up 1 */
                    if (dim && val) {
                        const double u1 = unit_open_left(orc_splitmix64(seed, ctr + 1));
                        const double u2 = unit_open_right(orc_splitmix64(seed, ctr + 2));
                        const double g = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
                        dim[nnz] = i;
                        val[nnz] = (float)g;
                    }
                    ++nnz;
                }
            }
        }
    }
    col_off[T * l] = (int32_t)nnz;
    return nnz;
}

/*
 * Number of nonzeros per vector in the fixed-count variant: ceil(a d),
 * clamped to [1, d].  a arrives as a float, so a*d is computed in double with
 * a relative allowance of 1e-6 (1/sqrt(784) as a float times 784 is
 * 28.0000013, meant as 28).
 */
int32_t orc_fixed_count(float density, int32_t d)
{
    double k = ceil((double)density * (double)d * (1.0 - 1e-6));
    if (k < 1.0) k = 1.0;
    if (k > (double)d) k = (double)d;
    return (int32_t)k;
}

typedef struct { double z; int32_t i; } draw_dim;

static int cmp_draw_dim(const void *pa, const void *pb)
{
    const draw_dim *a = (const draw_dim *)pa, *b = (const draw_dim *)pb;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

static int cmp_i32(const void *pa, const void *pb)
{
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/*
 * The ablation in the footnote of Sec. II-D: every vector has exactly
 * k = orc_fixed_count(density, d) nonzeros instead of a Bernoulli(a) draw per
 * component.  Reading: column c's nonzero dimensions are the k dimensions
 * with the smallest (z_i, i), where z_i is the same uniform draw (counter
 * 3(c d + i)) that the Bernoulli variant compares with a -- a uniformly
 * random k-subset -- and their values are the same Box-Muller normals
 * (counters 3(c d + i) + 1, + 2).  Output as in orc_random_matrix (always
 * T*l*k nonzeros; dim and val may be NULL).
 */
int64_t orc_random_matrix_fixed(int32_t T, int32_t l, int32_t d, float density, uint64_t seed,
                                int32_t *col_off, int32_t *dim, float *val)
{
    const int32_t k = orc_fixed_count(density, d);
    const double two_pi = 2.0 * 3.14159265358979323846;
    draw_dim *dd = (draw_dim *)malloc(sizeof(draw_dim) * (size_t)d);
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    int64_t nnz = 0;
    for (int32_t c = 0; c < T * l; ++c) {
        col_off[c] = (int32_t)nnz;
        if (dim && val) {
            for (int32_t i = 0; i < d; ++i) {
                const uint64_t ctr = 3ULL * (((uint64_t)c * (uint64_t)d) + (uint64_t)i);
                dd[i].z = unit_open_right(orc_splitmix64(seed, ctr));
                dd[i].i = i;
            }
            qsort(dd, (size_t)d, sizeof(draw_dim), cmp_draw_dim);
            for (int32_t r = 0; r < k; ++r) pick[r] = dd[r].i;
            qsort(pick, (size_t)k, sizeof(int32_t), cmp_i32);
            for (int32_t r = 0; r < k; ++r) {
                const uint64_t ctr = 3ULL * (((uint64_t)c * (uint64_t)d) + (uint64_t)pick[r]);
                const double u1 = unit_open_left(orc_splitmix64(seed, ctr + 1));
                const double u2 = unit_open_right(orc_splitmix64(seed, ctr + 2));
                dim[nnz + r] = pick[r];
                val[nnz + r] = (float)(sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
            }
        }
        nnz += k;
    }
    col_off[T * l] = (int32_t)nnz;
    free(dd);
    free(pick);
    return nnz;
}

/* --------------------------------------------------------- projection ---- */

/* One projection: sum over the column's nonzeros in ascending dimension, each
 * step a single rounding fmaf, starting from +0.0f. */
static float project_one(const float *x, int32_t c, const int32_t *col_off,
                         const int32_t *dim, const float *val)
{
    float acc = 0.0f;
    for (int32_t e = col_off[c]; e < col_off[c + 1]; ++e)
        acc = fmaf(x[dim[e]], val[e], acc);
    return acc;
}

/* P = X R (Algorithm 1) for all `ncols` columns; P is n x ncols row-major. */
void orc_project(const float *X, int64_t n, int32_t d, int32_t ncols,
                 const int32_t *col_off, const int32_t *dim, const float *val, float *P)
{
    for (int64_t x = 0; x < n; ++x)
        for (int32_t c = 0; c < ncols; ++c)
            P[x * ncols + c] = project_one(X + x * d, c, col_off, dim, val);
}

/* ------------------------------------------------------- tree growth ---- */

typedef struct { float key; int32_t id; } keyed;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct {
    const float *P;
    int32_t ncols, col0, l;
    float *split;
    int32_t *leaf_off, *leaf_ids;
    int32_t next_leaf, written;
    keyed *scratch;
} grow_ctx;

/* Algorithm 2.  `idx` holds the c member ids of heap node `node` at `level`. */
static void grow(grow_ctx *g, int32_t *idx, int32_t c, int32_t level, int64_t node)
{
    if (level == g->l) { /* a leaf: store its points, ids ascending */
        qsort(idx, (size_t)c, sizeof(int32_t), cmp_i32);
        g->leaf_off[g->next_leaf] = g->written;
        memcpy(g->leaf_ids + g->written, idx, (size_t)c * sizeof(int32_t));
        g->written += c;
        g->next_leaf += 1;
        g->leaf_off[g->next_leaf] = g->written;
        return;
    }
    /* proj <- P[indices, level]; order the points by (projection, id) */
    for (int32_t i = 0; i < c; ++i) {
        g->scratch[i].key = g->P[(int64_t)idx[i] * g->ncols + g->col0 + level];
        g->scratch[i].id = idx[i];
    }
    qsort(g->scratch, (size_t)c, sizeof(keyed), cmp_keyed);
    /* the first ceil(c/2) points in that order go left (Sec. II-A) and the
     * split value is the projection of the last of them (the median) */
    const int32_t nl = (c + 1) / 2;
    g->split[node] = g->scratch[nl - 1].key;
    for (int32_t i = 0; i < c; ++i) idx[i] = g->scratch[i].id;
    grow(g, idx, nl, level + 1, 2 * node + 1);
    grow(g, idx + nl, c - nl, level + 1, 2 * node + 2);
}

/*
 * Grow one tree of depth l over points 0..n-1 whose level-j projection is
 * P[x*ncols + col0 + j].  Writes split[2^l - 1] (heap order: children of node
 * h are 2h+1, 2h+2), leaf_off[2^l + 1] and leaf_ids[n] (leaves left to right,
 * ids ascending within a leaf).  Returns 0, or -1 if 2^l > n or n < 1.
 */
int32_t orc_grow_tree(const float *P, int64_t n, int32_t ncols, int32_t col0, int32_t l,
                      float *split, int32_t *leaf_off, int32_t *leaf_ids)
{
    if (n < 1 || l < 0 || l > 30 || ((int64_t)1 << l) > n) return -1;
    grow_ctx g;
    g.P = P; g.ncols = ncols; g.col0 = col0; g.l = l;
    g.split = split; g.leaf_off = leaf_off; g.leaf_ids = leaf_ids;
    g.next_leaf = 0; g.written = 0;
    g.scratch = (keyed *)malloc((size_t)n * sizeof(keyed));
    int32_t *idx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!g.scratch || !idx) { free(g.scratch); free(idx); return -2; }
    for (int64_t i = 0; i < n; ++i) idx[i] = (int32_t)i;
    grow(&g, idx, (int32_t)n, 0, 0);
    free(idx);
    free(g.scratch);
    return 0;
}

/* ----------------------------------------------------------- routing ---- */

/* Algorithm 3: descend l levels, p[level] <= split goes left.  p holds the
 * tree's l projections of the query.  Returns the leaf number 0..2^l-1. */
int32_t orc_route(const float *p, const float *split, int32_t l)
{
    int64_t node = 0;
    for (int32_t level = 0; level < l; ++level)
        node = (p[level] <= split[node]) ? 2 * node + 1 : 2 * node + 2;
    return (int32_t)(node - (((int64_t)1 << l) - 1));
}

/* ------------------------------------------------------------ voting ---- */

/*
 * Algorithm 4's vote loop for one query.  leaf_of_q[t] is the query's leaf
 * in tree t; leaf_off is T x (L+1), leaf_ids is T x n.  votes[n] receives
 * F(x; q) (Sec. III-A); cand (capacity n, may be NULL) receives S in the
 * order in which points reach v votes.  Returns |S|.
 */
int64_t orc_votes(int32_t T, int64_t n, int32_t L, const int32_t *leaf_of_q,
                  const int32_t *leaf_off, const int32_t *leaf_ids, int32_t v,
                  int32_t *votes, int32_t *cand)
{
    int64_t s = 0;
    for (int64_t x = 0; x < n; ++x) votes[x] = 0;
    for (int32_t t = 0; t < T; ++t) {
        const int32_t *off = leaf_off + (int64_t)t * (L + 1);
        const int32_t *ids = leaf_ids + (int64_t)t * n;
        const int32_t leaf = leaf_of_q[t];
        for (int32_t e = off[leaf]; e < off[leaf + 1]; ++e) {
            const int32_t point = ids[e];
            votes[point] += 1;
            if (votes[point] == v) {
                if (cand) cand[s] = point;
                ++s;
            }
        }
    }
    return s;
}

/* ------------------------------------------------------- exact search ---- */

typedef struct { double dist; int32_t id; } scored;

static int cmp_scored(const void *pa, const void *pb)
{
    const scored *a = (const scored *)pa, *b = (const scored *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Squared Euclidean distance (Sec. I-A) in double (mode 0) or in float,
 * summed sequentially over i with no fused operations (mode 1). */
static double sq_dist(const float *q, const float *x, int32_t d, int32_t mode)
{
    if (mode == 0) {
        double acc = 0.0;
        for (int32_t i = 0; i < d; ++i) {
            const double diff = (double)q[i] - (double)x[i];
            acc += diff * diff;
        }
        return acc;
    }
    float acc = 0.0f;
    for (int32_t i = 0; i < d; ++i) {
        const float diff = q[i] - x[i];
        const float sq = diff * diff;
        acc = acc + sq;
    }
    return (double)acc;
}

/* knn(q, k, S): the k points of S nearest to q, ordered by (distance, id);
 * out_dists holds Euclidean distances; missing entries are (-1, +inf). */
static void knn_on_set(const float *X, int32_t d, const float *q, const int32_t *S, int64_t s,
                       int32_t k, int32_t mode, scored *buf, int32_t *out_ids, float *out_dists)
{
    for (int64_t e = 0; e < s; ++e) {
        buf[e].id = S[e];
        buf[e].dist = sq_dist(q, X + (int64_t)S[e] * d, d, mode);
    }
    qsort(buf, (size_t)s, sizeof(scored), cmp_scored);
    for (int32_t r = 0; r < k; ++r) {
        if (r < s) {
            out_ids[r] = buf[r].id;
            out_dists[r] = (mode == 0) ? (float)sqrt(buf[r].dist) : sqrtf((float)buf[r].dist);
        } else {
            out_ids[r] = -1;
            out_dists[r] = INFINITY;
        }
    }
}

int32_t orc_knn(const float *X, int32_t d, const float *q, const int32_t *S, int64_t s,
                int32_t k, int32_t mode, int32_t *out_ids, float *out_dists)
{
    scored *buf = (scored *)malloc((size_t)(s > 0 ? s : 1) * sizeof(scored));
    if (!buf) return -2;
    knn_on_set(X, d, q, S, s, k, mode, buf, out_ids, out_dists);
    free(buf);
    return 0;
}

static void set_threads(int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Algorithm 4 for m queries.  The index is the output of orc_random_matrix
 * (R, T*l columns) and of orc_grow_tree for every tree: split is T x (L-1),
 * leaf_off is T x (L+1), leaf_ids is T x n.  Only the first `T` trees are
 * used.  Optional outputs (NULL to skip): out_proj m x (T*l), out_leaf m x T,
 * out_ncand m.  Queries are independent; with nthreads > 1 they are spread
 * over OpenMP threads, each running the same sequential steps.
 */
int32_t orc_query(const float *X, int64_t n, int32_t d, int32_t T, int32_t l,
                  const int32_t *col_off, const int32_t *dim, const float *val,
                  const float *split, const int32_t *leaf_off, const int32_t *leaf_ids,
                  const float *Q, int64_t m, int32_t k, int32_t v, int32_t mode, int32_t nthreads,
                  int32_t *out_ids, float *out_dists,
                  float *out_proj, int32_t *out_leaf, int64_t *out_ncand)
{
    const int32_t L = 1 << l;
    const int32_t ncols = T * l;
    int32_t status = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        float *p = (float *)malloc((size_t)(ncols > 0 ? ncols : 1) * sizeof(float));
        int32_t *leaf_of_q = (int32_t *)malloc((size_t)T * sizeof(int32_t));
        int32_t *votes = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        int32_t *S = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        scored *buf = (scored *)malloc((size_t)n * sizeof(scored));
        if (!p || !leaf_of_q || !votes || !S || !buf) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t qi = 0; qi < m; ++qi) {
                const float *q = Q + qi * d;
                /* tree_query (Algorithm 3): project, then route in every tree */
                for (int32_t c = 0; c < ncols; ++c)
                    p[c] = project_one(q, c, col_off, dim, val);
                for (int32_t t = 0; t < T; ++t)
                    leaf_of_q[t] = orc_route(p + t * l, split + (int64_t)t * (L - 1), l);
                /* voting (Algorithm 4), then knn(q, k, S) */
                const int64_t s = orc_votes(T, n, L, leaf_of_q, leaf_off, leaf_ids, v, votes, S);
                knn_on_set(X, d, q, S, s, k, mode, buf, out_ids + qi * k, out_dists + qi * k);
                if (out_proj) memcpy(out_proj + qi * ncols, p, (size_t)ncols * sizeof(float));
                if (out_leaf) memcpy(out_leaf + qi * T, leaf_of_q, (size_t)T * sizeof(int32_t));
                if (out_ncand) out_ncand[qi] = s;
            }
        }
        free(p); free(leaf_of_q); free(votes); free(S); free(buf);
    }
    return status;
}

/* Exact k-NN (Sec. I-A) over all n points, double precision, ordered by
 * (distance, id).  Ground truth for recall. */
int32_t orc_brute_knn(const float *X, int64_t n, int32_t d, const float *Q, int64_t m,
                      int32_t k, int32_t nthreads, int32_t *out_ids, float *out_dists)
{
    int32_t status = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        scored *buf = (scored *)malloc((size_t)n * sizeof(scored));
        if (!buf) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t qi = 0; qi < m; ++qi) {
                const float *q = Q + qi * d;
                for (int64_t x = 0; x < n; ++x) {
                    buf[x].id = (int32_t)x;
                    buf[x].dist = sq_dist(q, X + x * d, d, 0);
                }
                qsort(buf, (size_t)n, sizeof(scored), cmp_scored);
                for (int32_t r = 0; r < k; ++r) {
                    if (r < n) {
                        out_ids[qi * k + r] = buf[r].id;
                        out_dists[qi * k + r] = (float)sqrt(buf[r].dist);
                    } else {
                        out_ids[qi * k + r] = -1;
                        out_dists[qi * k + r] = INFINITY;
                    }
                }
            }
        }
        free(buf);
    }
    return status;
}
