/*
 * mrpt.h -- C ABI of the GB300 (sm_103a) implementation of multiple random
 * projection trees with voting (Hyvonen et al., "Fast k-NN search",
 * arXiv:1509.06957).
 *
 * Offline phase (Sec. I-A, Sec. II, Algorithms 1-2): mrpt_build grows T
 * sparse random projection trees of depth l over n points of dimension d.
 * Online phase (Sec. III, Algorithms 3-4): mrpt_query routes each query down
 * every tree, counts votes over the T leaves it lands in, keeps the points
 * with at least v votes as the candidate set S and returns the k nearest
 * members of S by Euclidean distance.
 *
 * Conventions shared by every entry point:
 *   - All matrices are row-major, float32, tightly packed (row stride = d).
 *   - Pointer arguments may be host or device memory of the current CUDA
 *     device; the library asks the CUDA runtime which.  Device buffers are
 *     used in place.  Host buffers (pinned or pageable) are staged through
 *     device buffers owned by the index, and a call that was given any host
 *     buffer returns only after its results are in that buffer.  Host
 *     queries in batches of 8,192 or more are copied in four chunks on a
 *     second stream owned by the index, each chunk routed as it arrives
 *     (pinned memory lets the copies overlap the routing).
 *   - A call given only device buffers is stream-ordered on the index's
 *     stream (mrpt_set_stream) and may return before the GPU has finished.
 *     Errors detected on the device (a non-finite query value) are latched
 *     in the index and reported by mrpt_sync or by the next call that
 *     synchronises.
 *   - Return value: MRPT_OK (0) or a negative MRPT_ERR_* code; after an
 *     error, mrpt_last_error() gives a message for the calling thread.
 *   - One index may be used by one host thread at a time, and queries on one
 *     index run one after another (they share the index's scratch buffers).
 *   - Ids are int32: n < 2^31.
 */
#ifndef MRPT_H
#define MRPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRPT_OK 0
#define MRPT_ERR_INVALID_ARG -1      /* a size, parameter or pointer is out of range */
#define MRPT_ERR_NONFINITE_INPUT -2  /* NaN or Inf in the data or in a query */
#define MRPT_ERR_OOM -3              /* a device or host allocation failed */
#define MRPT_ERR_CUDA -4             /* a CUDA runtime call failed */
#define MRPT_ERR_TIMEOUT -5          /* a bounded device-side wait ran out */
#define MRPT_ERR_UNSUPPORTED -6      /* valid request outside this build's limits */

/* Limits of this build. */
#define MRPT_MAX_TREES 255   /* vote counters are 8-bit; F(x;q) <= T (Sec. III-A) */
#define MRPT_MAX_DEPTH 24    /* 2^l leaves per tree */
#define MRPT_MAX_K 256       /* neighbours per query */
#define MRPT_MAX_DIM 32768   /* dimension d */

typedef struct mrpt_index mrpt_index; /* opaque; owned by the library */

/*
 * mrpt_build -- Algorithm 1 (grow T trees) with Algorithm 2 per tree.
 *
 *   data     n x d float32, host or device; copied into memory owned by the
 *            index, so the caller may free it when the call returns.
 *   n, d     number of points (2^l <= n < 2^31) and dimension (1..MRPT_MAX_DIM).
 *   T        number of trees, 1..MRPT_MAX_TREES.
 *   l        depth, 0..MRPT_MAX_DEPTH, with 2^l <= n.  Leaves hold
 *            ceil(n/2^l) or floor(n/2^l) points (Sec. III-A).
 *   density  the paper's sparsity a in (0, 1] (Sec. II-B); each component
 *            of each level's random vector is N(0,1) with probability a,
 *            else 0.  a = 1/sqrt(d) is the paper's choice; 0 or a negative
 *            value selects it.
 *   seed     key of the counter-based random source: component i of tree
 *            t's level-j vector takes draws 3((t l + j) d + i) + {0,1,2} of
 *            SplitMix64 started at `seed` (Bernoulli by u < a, N(0,1) by
 *            Box-Muller in double, rounded to float).  Trees are therefore
 *            prefix-stable: the first T trees of a larger index are equal.
 *   out      receives the new index.
 *
 * Points are split at the median of their projections with the order-based
 * rule of Sec. II-A: sorted by (projection, id), the first ceil(c/2) points
 * of a node go left and the node's split value is the projection of the
 * last of them.  Projections are fmaf chains over each vector's nonzeros in
 * ascending dimension from +0.0f (one rounding per term).
 * Errors: INVALID_ARG, NONFINITE_INPUT (data holds NaN/Inf), OOM, CUDA.
 * Synchronous: returns after the index is complete.
 */
int mrpt_build(const float *data, int64_t n, int32_t d, int32_t T, int32_t l, float density,
               uint64_t seed, mrpt_index **out);

/*
 * mrpt_build_ex -- mrpt_build with options (opts may be NULL: the defaults).
 *
 *   sparsity  how each level's random vector gets its nonzeros:
 *     MRPT_SPARSITY_BERNOULLI (0, default): component i is nonzero with
 *       probability density (Sec. II-B), as in mrpt_build.
 *     MRPT_SPARSITY_FIXED (1): exactly ceil(density * d) nonzeros per vector
 *       (at least 1, at most d; density * d is taken with a relative
 *       allowance of 1e-6, since density is a float) -- the variant in the
 *       footnote of Sec. II-D, an ablation of Table III.  The nonzero
 *       dimensions are those with the smallest (first draw, dimension), the
 *       first draw being the one the Bernoulli rule compares with density,
 *       so the set is a uniformly random subset; values are the same N(0,1)
 *       draws as in the Bernoulli rule.
 * Errors: those of mrpt_build; INVALID_ARG for an unknown sparsity or a tree
 * offset out of range.
 */
#define MRPT_SPARSITY_BERNOULLI 0
#define MRPT_SPARSITY_FIXED 1

typedef struct mrpt_build_opts {
    int32_t sparsity;
    int32_t tree_offset;  /* t0 >= 0, t0 + T <= MRPT_MAX_TREES: the index holds trees t0 ..
                             t0+T-1 of the random source (tree i of the index takes the
                             draws of tree t0+i), so it equals trees t0.. of an index of
                             t0+T trees with the same seed -- one shard of a tree-sharded
                             index (Sec. I-C: the trees are independent and may live on
                             different machines).  0 (default): trees 0..T-1. */
} mrpt_build_opts;

int mrpt_build_ex(const float *data, int64_t n, int32_t d, int32_t T, int32_t l, float density,
                  uint64_t seed, const mrpt_build_opts *opts, mrpt_index **out);

/*
 * mrpt_query -- Algorithm 4 (with Algorithm 3 per tree) for m queries.
 *
 *   Q          m x d float32 queries, host or device.
 *   m          number of queries, >= 0 (0 is a no-op).
 *   k          neighbours per query, 1..MRPT_MAX_K.
 *   v          vote threshold, 1..T: S = {x : F(x;q) >= v} (Sec. III-A).
 *   out_ids    m x k int32: row i holds query i's neighbours ordered by
 *              (distance, id) ascending; -1 where |S| < k.
 *   out_dists  m x k float32 Euclidean distances (Sec. I-A), +inf where
 *              |S| < k.  Distances are accumulated in float32.
 * The default path keeps each query's S in a device list of
 * T ceil(n/2^l) / v entries (at most n), the most S can hold (Sec. III-B), and
 * splits the exact search on S into chunks that warps take in turn; when the
 * lists of the whole batch would take more than 2 GiB the batch runs as
 * consecutive sub-batches.  The scratch stays with the index for later calls.
 * Equivalent to mrpt_query_ex with opts = NULL.
 * Errors: INVALID_ARG, NONFINITE_INPUT (latched, see above), OOM, CUDA.
 */
int mrpt_query(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
               int32_t *out_ids, float *out_dists);

/* Optional controls and debug outputs of mrpt_query_ex.  Zero-initialise
 * and set what is needed.  Debug pointers are device or host buffers. */
typedef struct mrpt_query_opts {
    int32_t n_trees;      /* use the first n_trees trees (0 = all T) */
    int32_t path;         /* 0: vote/emit kernel + candidate-search kernel (default);
                             1: one fused vote + search kernel.  Same results. */
    int32_t precision;    /* MRPT_PREC_FP32 (0, default), MRPT_PREC_BF16 (1) or
                             MRPT_PREC_FP8 (2): candidate distances from the index's
                             reduced-precision copy (mrpt_add_lowp), accumulated in
                             float32; the k + margin nearest by that distance are then
                             re-ranked with exact float32 distances.  When the bfloat16
                             copy is lossless (every value exactly a bfloat16) those
                             distances are the float32 ones up to summation order and
                             the re-rank is skipped.  Path 0 only. */
    int32_t margin;       /* survivors beyond k kept for the re-rank (k + margin <= 256) */
    int32_t chunk;        /* tuning, path 0: candidates per search work item (0 = auto) */
    int32_t ring;         /* tuning, path 0: candidate rows staged per search warp, 2..16
                             (0 = auto) */
    /* debug outputs (NULL = not written) */
    float *proj;          /* m x (n_trees*l): p = q^T R per tree and level (Algorithm 3) */
    int32_t *leaf;        /* m x n_trees: the query's leaf in each tree */
    uint8_t *votes;       /* m x n: F(x;q) per point (Sec. III-A) */
    int64_t *n_cand;      /* m: |S| */
    int32_t *cand;        /* m x cand_cap: members of S (any order) */
    int64_t cand_cap;     /* row capacity of `cand`; members past it are dropped */
    /* host float[4] (NULL = not measured): device time in ms of routing,
     * of voting (path 0: the vote/emit kernel; path 1: the fused kernel), of
     * the candidate search (path 0; 0 for path 1) and of the whole query,
     * from CUDA events recorded on the index's stream; the call then
     * synchronises */
    float *stage_ms;
    /* path 0: how a query's votes are counted (Sec. III-A: F(x;q) for the
     * points of its T leaves).  0 (default) and 1: 8-bit counters in shared
     * memory, over 65,536-id chunks (one pass per chunk) when n > 65,536.
     * 2: one pass over a hash table of (id, count) words in shared memory;
     * INVALID_ARG when n_trees * ceil(n / 2^l) exceeds
     * MRPT_VOTE_HASH_ENTRIES or n >= 2^24.  Same results. */
    int32_t vote_table;
} mrpt_query_opts;

#define MRPT_VOTE_COUNTERS 1
#define MRPT_VOTE_HASH 2
/* entries of a query's T leaves the hash table takes: 3/4 of its 32,768
 * slots, so the table never fills */
#define MRPT_VOTE_HASH_ENTRIES 24576

int mrpt_query_ex(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
                  const mrpt_query_opts *opts, int32_t *out_ids, float *out_dists);

#define MRPT_PREC_FP32 0
#define MRPT_PREC_BF16 1
#define MRPT_PREC_FP8 2

/*
 * mrpt_add_lowp -- add a reduced-precision copy of the data to the index for
 * the candidate distances of later queries (mrpt_query_opts.precision):
 * the exact search knn(q, k, S) of Algorithm 4 on fewer bytes per row.  The
 * paper states no precision (Sec. IV-B); this copy has no counterpart there,
 * and the float32 re-rank restores the exact order of the survivors.
 * MRPT_PREC_BF16: every value rounded to bfloat16 (nearest even), same row
 * layout, 2 bytes per value.  MRPT_PREC_FP8: each row scaled by
 * 448 / max|x| and rounded to e4m3 (saturating), 1 byte per value plus the
 * row's float32 scale (rows padded to 16 bytes).  The float32 data stays in
 * the index for the re-rank.  Synchronous.  Errors: INVALID_ARG, OOM, CUDA.
 */
int mrpt_add_lowp(mrpt_index *idx, int32_t precision);

/*
 * Query plans: the whole query (counter clears and every kernel) captured
 * once into a CUDA graph and replayed per batch, which removes the per-call
 * launch work for streams of small, uneven batches.  They compute exactly
 * Algorithms 3-4 as mrpt_query does; the paper has no counterpart (it runs
 * one query at a time on a CPU, Sec. IV).  A plan fixes k, v and
 * the options (n_trees, path, precision, margin, chunk, ring; debug outputs
 * and stage_ms are not available) and a largest batch m_max; it owns its
 * scratch, so plans of one index may run on different streams.  The kernels
 * read each batch's query pointer, output pointers and size from a small
 * device record, so one graph serves every m <= m_max.
 *
 * mrpt_plan_create -- capture the plan (synchronous; allocates).
 * mrpt_plan_run    -- answer m <= m_max queries, exactly as mrpt_query_ex
 *                     with the plan's options.  Buffers may be host or device
 *                     memory (host buffers are staged; the call then returns
 *                     after the results are in place).  Runs on the index's
 *                     stream at the time of the call.
 * mrpt_plan_free   -- release the plan (NULL is accepted).
 * Errors: INVALID_ARG, OOM, CUDA (and as mrpt_query).
 */
typedef struct mrpt_plan mrpt_plan;
int mrpt_plan_create(mrpt_index *idx, int64_t m_max, int32_t k, int32_t v,
                     const mrpt_query_opts *opts, mrpt_plan **out);
int mrpt_plan_run(mrpt_plan *plan, const float *Q, int64_t m, int32_t *out_ids,
                  float *out_dists);
int mrpt_plan_free(mrpt_plan *plan);

/*
 * mrpt_save / mrpt_load -- the index in the compact form that a median split
 * allows (Sec. II-A): header, the random matrix (compressed columns), one
 * split value per inner node, the leaf lists and the data; leaf boundaries
 * are not stored (they follow from n and l).  Host byte order.  A loaded index
 * answers queries exactly as the saved one; reduced-precision copies are not
 * saved (call mrpt_add_lowp again).  Synchronous.
 * Errors: INVALID_ARG (path, bad or truncated file), OOM, CUDA.
 */
int mrpt_save(const mrpt_index *idx, const char *path);
int mrpt_load(const char *path, mrpt_index **out);

/* Release the index and everything it owns.  NULL is accepted.
 * (Housekeeping: no counterpart in the paper.) */
int mrpt_free(mrpt_index *idx);

/* Message of the calling thread's last error ("" if none).
 * (Housekeeping: no counterpart in the paper.) */
const char *mrpt_last_error(void);

/* Stream on which the index's work is ordered (a cudaStream_t; NULL is the
 * legacy default stream).  Applies to later calls.
 * (Housekeeping: no counterpart in the paper.) */
int mrpt_set_stream(mrpt_index *idx, void *stream);

/* Wait for the index's stream, then report and clear the device-latched
 * status: MRPT_OK or MRPT_ERR_NONFINITE_INPUT / MRPT_ERR_TIMEOUT.
 * (Housekeeping: no counterpart in the paper.) */
int mrpt_sync(mrpt_index *idx);

/* Shape of an index: n, d (Sec. I-A), T, l, a (Sec. II-B), the seed, the
 * nonzeros of R and the device memory held. */
typedef struct mrpt_index_info {
    int64_t n;
    int32_t d, T, l;
    float density;
    uint64_t seed;
    int64_t nnz;           /* nonzeros of R over all T*l vectors */
    int64_t device_bytes;  /* device memory held (index + scratch) */
    int32_t tree_offset;   /* first tree of the random source held (mrpt_build_opts) */
} mrpt_index_info;

int mrpt_info(const mrpt_index *idx, mrpt_index_info *info);

/* Index contents, for inspection and tests: the random vectors
 * (Algorithm 1), the split values and leaves (Algorithm 2). */
enum mrpt_export_what {
    MRPT_EXPORT_R_COL_OFF = 0, /* int32 [T*l+1] column offsets of R (column t*l+j) */
    MRPT_EXPORT_R_DIM = 1,     /* int32 [nnz] dimension of each nonzero, ascending per column */
    MRPT_EXPORT_R_VAL = 2,     /* float32 [nnz] value of each nonzero */
    MRPT_EXPORT_SPLIT = 3,     /* float32 [T][2^l-1] split values, heap order per tree */
    MRPT_EXPORT_LEAF_OFF = 4,  /* int32 [T][2^l+1] leaf offsets into LEAF_IDS rows */
    MRPT_EXPORT_LEAF_IDS = 5,  /* int32 [T][n] point ids, leaves left to right, ids ascending */
    MRPT_EXPORT_DATA = 6       /* float32 [n][d] the index's copy of the data */
};

/* Bytes that mrpt_export writes for `what` (negative error code if invalid);
 * the parts are those of Algorithms 1-2 listed above. */
int64_t mrpt_export_size(const mrpt_index *idx, int32_t what);

/* Copy `what` (a part of the index of Algorithms 1-2, listed above) into
 * dst (host or device, dst_bytes >= mrpt_export_size).  Synchronous. */
int mrpt_export(const mrpt_index *idx, int32_t what, void *dst, int64_t dst_bytes);

/*
 * mrpt_query_noalloc -- mrpt_query that allocates nothing.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *
 * mrpt_query grows scratch buffers with cudaMalloc on first use.  Callers
 * that cannot allocate -- a serving loop with a latency budget (cudaMalloc
 * and cudaFree may synchronise the device), or a process whose device
 * memory is owned or capped by another framework's pool -- use this entry
 * point instead.  It runs the same kernels; its scratch (the leaf of each
 * query in each tree, and the counter that hands queries to blocks) lives in
 * one fixed 4 MiB array that every GPU loading this library holds until the
 * process exits.
 *
 *   Q, out_ids, out_dists   device memory only (m x d, m x k, m x k), as in
 *                           mrpt_query; host pointers are rejected.
 *   n_trees                 use the first n_trees trees (0 = all T).
 *   limit                   m * n_trees <= MRPT_NOALLOC_MAX_LEAF_ENTRIES;
 *                           larger batches are rejected with INVALID_ARG
 *                           (split the batch).
 * The first call on a device looks up the array's device address (once per
 * device, under a lock); make that first call before any stream capture.
 * Every call, from any index or stream, shares the one array: the work
 * counter is cleared at the start of each call, and calls whose GPU work
 * overlaps in time race on the array.  Stream-ordered on the index's stream;
 * no device-side status is latched beyond mrpt_query's (see mrpt_sync).
 * Errors: INVALID_ARG, CUDA.
 */
#define MRPT_NOALLOC_MAX_LEAF_ENTRIES 1048512 /* (4 MiB - 256 B) / 4 */
int mrpt_query_noalloc(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
                       int32_t n_trees, int32_t *out_ids, float *out_dists);

/*
 * Tree-sharded voting (Sec. I-C: the trees of an index are independent, so
 * they can be spread over machines).  Build one index per shard with
 * mrpt_build_opts.tree_offset (shard g holds trees t_g .. t_g + T_g - 1 of
 * one seed), count each query's votes among the local trees with
 * mrpt_vote_counts, exchange the lists (any transport), and answer each
 * query on the shard that owns it with mrpt_query_from_counts.  F(x;q) is
 * the sum of the shards' counts and S = {x : F >= v} (Sec. III-A), so the
 * rows are those of one index that holds all the trees.
 *
 * mrpt_vote_counts -- for each of the m queries, every id with at least one
 * vote among the index's first n_trees trees (0 = all) and its count, ids
 * ascending.
 *   Q           m x d float32, device memory.
 *   cap         row capacity of out_ids and out_counts, at least
 *               min(n_trees ceil(n / 2^l), n), the most ids a query can meet.
 *   out_nnz     int32 [m]: ids written for each query.
 *   out_ids     int32 [m x cap]: row i's first out_nnz[i] entries.
 *   out_counts  uint8 [m x cap]: their counts (1 .. n_trees).
 * Every buffer is device memory; stream-ordered on the index's stream.
 * Errors: INVALID_ARG (cap below the bound, given in the message; a host
 * buffer), OOM, CUDA.
 */
int mrpt_vote_counts(mrpt_index *idx, const float *Q, int64_t m, int32_t n_trees, int64_t cap,
                     int32_t *out_nnz, int32_t *out_ids, uint8_t *out_counts);

/*
 * mrpt_query_from_counts -- Algorithm 4 from vote counts gathered from the
 * shards: query i's (id, count) pairs are entries off[i] .. off[i+1]-1 of
 * ids and counts, in any order and with an id repeated once per shard.
 * F(x;q) is the sum of x's counts; it must stay within 255, which holds for
 * disjoint shards of MRPT_MAX_TREES trees in all.  S = {x : F >= v} and the
 * rows are those of mrpt_query: the k nearest members of S by (distance,
 * id), padded with (-1, +inf).  Ids outside [0, n) are ignored.
 *   Q           m x d float32 queries.
 *   off         int64 [m+1], non-decreasing from 0.
 *   v           1 .. MRPT_MAX_TREES.
 *   opts        NULL or options: precision, margin, chunk and ring as in
 *               mrpt_query_ex (the other fields are ignored).
 *   out_ids, out_dists   m x k.
 * Every buffer is device memory.  The call copies off to the host and waits
 * for it, then runs stream-ordered on the index's stream.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int mrpt_query_from_counts(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
                           const int64_t *off, const int32_t *ids, const uint8_t *counts,
                           const mrpt_query_opts *opts, int32_t *out_ids, float *out_dists);

/* Fault injection for tests: make the allocation after the next `after`
 * successful ones fail with MRPT_ERR_OOM (negative disables).  Host-side
 * only; process-wide.  (Testing aid: no counterpart in the paper.) */
int mrpt_debug_fail_alloc_after(int32_t after);

/* Fault injection for tests: each wait for a staged candidate row in the
 * candidate search's distance loop (path 0) gives up after `tries` tries
 * instead of about two million (negative restores the full bound).  Such
 * waits (an mbarrier phase completed by a bulk copy of a whole row) exist
 * only where the search copies whole rows: rows longer than 1,024 values,
 * and rows shorter than 32 float32, 64 bfloat16 or 113 e4m3 values; the
 * other rows are copied per lane with cp.async, whose per-thread waits
 * always complete, and this setting does not affect them.  A warp
 * whose wait gives up stops, sets the index's status to MRPT_ERR_TIMEOUT
 * (reported by mrpt_sync, or by a call given host buffers) and first waits,
 * with the full bound, for its row copies still in flight; the rows of the
 * queries it held are not written.  Applies to launches made after the
 * call, including plans created after it.  Process-wide; host-side
 * setting only.  (Testing aid: no counterpart in the paper.) */
int mrpt_debug_row_wait_tries(int32_t tries);

#ifdef __cplusplus
}
#endif

#endif /* MRPT_H */
