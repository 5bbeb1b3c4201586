// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mrpt.h"

namespace mrpt {

// ------------------------------------------------------------------ errors --

void set_error(const std::string &msg);
void clear_error();

// Returns MRPT_ERR_CUDA (and records where) when `e` is not cudaSuccess.
int cuda_fail(cudaError_t e, const char *what);

#define MRPT_CUDA_TRY(call)                                          \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::mrpt::cuda_fail(_e, #call);  \
    } while (0)

// Tries of each row wait in the candidate search's distance loop: the full
// bound unless a test has shortened it (mrpt_debug_row_wait_tries).
uint32_t debug_row_wait_tries();

// Device allocation through one gate so that tests can inject failures.
int dev_alloc(void **p, size_t bytes, const char *what);

// True when `p` is memory of some CUDA device (not host memory).
bool is_device_ptr(const void *p);

// Grow-only device scratch buffer.
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
    int ensure(size_t need, const char *what);
    void release();
};

// Device-latched status bits (index->status[0]).
enum : uint32_t {
    STATUS_NONFINITE_QUERY = 1u,
    STATUS_TIMEOUT = 2u,
};

}  // namespace mrpt

// The index.  Device arrays are owned; see mrpt.h for their meaning.
struct mrpt_index {
    int64_t n = 0;
    int32_t d = 0;
    int32_t dpad = 0;       // row stride of X in elements (multiple of 8)
    int32_t T = 0, l = 0;
    int64_t L = 1;          // leaves per tree
    float density = 0.f;
    uint64_t seed = 0;
    int64_t nnz = 0;
    int32_t tree_offset = 0;  // tree t of this index is tree tree_offset + t of the random source
    int device = 0;
    cudaStream_t stream = nullptr;

    float *X = nullptr;          // n x dpad, zero padded
    uint16_t *Xb = nullptr;      // optional bfloat16 copy of X (same stride)
    bool bf16_exact = false;     // every value of X is exactly representable in bfloat16
    unsigned char *X8 = nullptr; // optional e4m3 copy: row8_bytes per row (values, scale)
    int32_t row8_bytes = 0;
    int32_t *col_off = nullptr;  // T*l + 1
    int32_t *dim = nullptr;      // nnz
    float *val = nullptr;        // nnz
    int2 *dv = nullptr;          // (dimension, value bits) of the nonzeros, columns at even pairs
    int2 *rcol = nullptr;        // T*l: (first pair in dv, count) of each column
    float *split = nullptr;      // T x (L-1)
    int32_t *leaf_off = nullptr; // L + 1 (identical for every tree)
    int32_t *leaf_ids = nullptr; // T x n
    // Vote layout (only when n <= VOTE_CHUNK_IDS): leaf j of tree t starts at
    // int4 index t*vote_s4 + leaf_off4[j] and holds the leaf's ids, then the
    // sentinel id up to a multiple of 4; within each 256-entry window the ids
    // are placed so that each of a warp's eight vote reductions meets as many
    // distinct counter banks ((id >> 2) mod 32) as the window allows.
    int4 *leaf4 = nullptr;
    int32_t *leaf_off4 = nullptr; // L + 1
    int64_t vote_s4 = 0;          // int4s per tree
    int32_t vote_win = 0;         // 128-entry windows per leaf (the longest leaf)
    // n > VOTE_CHUNK_IDS: per (tree t, leaf j) the position in tree t's
    // leaf_ids row of the first id >= c * VOTE_CHUNK_IDS, c = 0 .. n_chunks
    // (c = n_chunks: the leaf's end), at chunk_bnd[(t L + j)(n_chunks + 1) + c]
    int32_t *chunk_bnd = nullptr;
    int32_t n_chunks = 0;
    uint32_t *status = nullptr;  // [0] latched status bits, [1] work counter

    std::vector<int32_t> h_col_off, h_dim;
    std::vector<float> h_val;

    // query scratch
    mrpt::Scratch q_leaf;    // m x T int32
    mrpt::Scratch q_stage;   // staged host queries (m x d)
    mrpt::Scratch o_stage;   // staged outputs (m x k ids + m x k dists)
    mrpt::Scratch dbg_stage; // staged debug outputs
    mrpt::Scratch q_cand;    // candidate lists, |S| per query, work items, partial lists
    mrpt::Scratch shard;     // tree-sharded voting: dense vote rows and search scratch

    int64_t device_bytes = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // stage timing (created on first use)
    // host-buffer queries in pipelined chunks: a copy stream and per-chunk
    // events (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pev[16] = {};
};

namespace mrpt {

// ------------------------------------------------------ build (mrpt_build.cu)

// Random matrix of Algorithm 1 on the host (counter-based SplitMix64 +
// Box-Muller); compressed columns, column c = t*l + j.  sparsity is
// MRPT_SPARSITY_BERNOULLI or MRPT_SPARSITY_FIXED (see mrpt_build_ex); tree t
// takes the draws of tree tree_offset + t.
void generate_random_matrix(int32_t T, int32_t l, int32_t d, float density, uint64_t seed,
                            int32_t sparsity, int32_t tree_offset, std::vector<int32_t> &col_off,
                            std::vector<int32_t> &dim, std::vector<float> &val);

// Nonzeros per vector of MRPT_SPARSITY_FIXED: ceil(density * d) in [1, d].
int32_t fixed_nonzeros(float density, int32_t d);

// Most work items (chunks of its candidate list) that the candidate search
// makes of one query; long lists get longer chunks.
constexpr int CAND_ITEMS_MAX = 128;

// Work items of the candidate search for a query with c candidates: chunks
// of item_size(c) consecutive list entries, at least `chunk` and at most
// CAND_ITEMS_MAX chunks per query (one item even when S is empty, so that
// the row gets its padding).  item_count(c) * item_size(c) >= c and every
// item holds at least one candidate when c > 0.
__host__ __device__ __forceinline__ int item_size(int c, int chunk) {
    const int per = (c + CAND_ITEMS_MAX - 1) / CAND_ITEMS_MAX;
    return chunk > per ? chunk : per;
}
__host__ __device__ __forceinline__ int item_count(int c, int csz) { return c == 0 ? 1 : (c + csz - 1) / csz; }

// Ids whose 8-bit vote counters fit in shared memory at once (64 KB).
constexpr int64_t VOTE_CHUNK_IDS = 65536;

// 32-bit words of 8-bit vote counters for the ids of one chunk (a multiple
// of 4 words); the word after them holds the sentinel's counter.
inline int32_t vote_cnt_words(int64_t n) {
    const int64_t ids = n < VOTE_CHUNK_IDS ? n : VOTE_CHUNK_IDS;
    return int32_t(((ids + 3) / 4 + 3) & ~int64_t(3));
}

// Id that pads a leaf of the vote layout (its counter is the word after the
// real ones; it is never reported as a candidate).
inline int32_t vote_sentinel(int64_t n) { return 4 * vote_cnt_words(n); }

// Builds idx->leaf4 / leaf_off4 from idx->leaf_ids, or for n above
// VOTE_CHUNK_IDS the id-chunk boundaries of every leaf (idx->chunk_bnd).
int build_vote_layout(mrpt_index *idx);

// Projections and median splits for every tree; fills idx->split,
// idx->leaf_off and idx->leaf_ids.  X, R must already be on the device.
int grow_trees_device(mrpt_index *idx);

// Leaf offsets (identical for every tree) of an index whose trees were loaded.
int compute_leaf_offsets(mrpt_index *idx);

// Sets *nonfinite when the n x dpad matrix X holds NaN/Inf.
int check_finite(const float *X, int64_t rows, int32_t stride, int32_t cols, cudaStream_t s,
                 bool *nonfinite);

// ------------------------------------------------------ query (mrpt_query.cu)

// One batch as a captured query graph sees it: the kernels read the query
// pointer, output pointers and batch size from this device-resident record
// (plan mode) instead of their launch arguments.
struct QueryRecord {
    const float *Q;
    int32_t *out_ids;
    float *out_dists;
    int64_t m;
};

struct QueryLaunch {
    const float *Q;        // m x d device queries
    int64_t m;
    int32_t k, v, n_trees;
    int32_t *out_ids;      // m x k device
    float *out_dists;      // m x k device
    float *proj;           // optional m x (n_trees*l)
    int32_t *leaf;         // m x n_trees device (scratch or debug)
    uint8_t *votes;        // optional m x n
    int64_t *n_cand;       // optional m
    int32_t *cand;         // optional m x cand_cap
    int64_t cand_cap;
    float *stage_ms;       // optional host float[4]
    const int64_t *cand_off; // optional: query i's candidate list starts at cand_list + cand_off[i]
                             // (instead of i * capq)
    int32_t path;          // 0: vote/emit + candidate search, 1: one fused kernel
    int32_t *cand_list;    // m x capq candidate lists (path 0)
    int32_t capq;          // >= |S| of any query: T ceil(n / 2^l) / v, at most n
    int32_t *ncand;        // m (path 0)
    int2 *items;           // m x max_items_q (query, chunk) work items (path 0)
    int32_t chunk;         // candidates per work item
    int32_t max_items_q;
    int32_t *done;         // m
    float *part_d;         // m x max_items_q x k partial top-k lists
    int32_t *part_i;
    int32_t precision;     // 0 float32 rows, 1 bfloat16 rows + float32 re-rank
    int32_t margin;        // survivors beyond k kept for the re-rank
    int32_t ring;          // candidate rows staged per search warp (0 = auto)
    int32_t vote_table;    // path 0: 0 auto, MRPT_VOTE_COUNTERS, MRPT_VOTE_HASH
    uint32_t *counters;    // 8 work-counter words ([0] unused); null = the index's
    cudaStream_t stream;   // stream of the launches (plans capture on their own)
    bool use_stream;       // take `stream` instead of the index's stream
    const QueryRecord *rec;  // plan mode: batch read on the device (m <= ql.m)
    bool routed;           // ql.leaf is already filled (routing skipped)
};

int launch_query(mrpt_index *idx, const QueryLaunch &ql);

// Routing alone (projection and descent) for ql.m queries into ql.leaf.
int launch_route_only(mrpt_index *idx, const QueryLaunch &ql);

// The candidate search alone (k_cand_knn): the candidate lists (ql.cand_list
// with ql.capq or ql.cand_off), |S| (ql.ncand), the work items and their
// counter (counter word 5) must already be written; counter word 2 must be 0.
int launch_search_only(mrpt_index *idx, const QueryLaunch &ql);

// launch_query with caller-supplied scratch: ql.leaf holds the m x n_trees
// leaf-of-query table and `work` the work counter.
int launch_query_with_counter(mrpt_index *idx, const QueryLaunch &ql, uint32_t *work);

// Fills idx->Xb with X rounded to bfloat16 (allocating it on first use).
int make_bf16_copy(mrpt_index *idx);

// Fills idx->X8 with X as e4m3 with a per-row scale (allocating it first).
int make_fp8_copy(mrpt_index *idx);

// Stream-ordered write of a plan's batch record.
int set_record(QueryRecord *rec, const QueryRecord &r, cudaStream_t s);

}  // namespace mrpt
