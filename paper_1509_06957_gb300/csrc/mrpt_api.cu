// C ABI (include/mrpt.h): argument checks, ownership, host/device staging.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <string>

#include "mrpt_internal.cuh"

namespace mrpt {

namespace {
thread_local std::string g_last_error;
// Scratch of the two-kernel path (candidate lists, work items, partial
// lists) that one launch may use; a batch that needs more runs in
// consecutive sub-batches.
constexpr size_t kCandScratchBudget = size_t(2) << 30;
std::atomic<int32_t> g_fail_after{-1};
std::atomic<int32_t> g_row_wait_tries{-1};
}  // namespace

uint32_t debug_row_wait_tries() {
    const int32_t t = g_row_wait_tries.load();
    return t < 0 ? (1u << 21) : uint32_t(t);
}

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return MRPT_ERR_CUDA;
}

static bool take_injected_failure() {
    int32_t cur = g_fail_after.load();
    while (cur >= 0) {
        if (g_fail_after.compare_exchange_weak(cur, cur - 1)) return cur == 0;
    }
    return false;
}

int dev_alloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (take_injected_failure()) {
        set_error(std::string("out of device memory (injected) allocating ") + what);
        return MRPT_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error(std::string("out of device memory allocating ") + what + " (" +
                  std::to_string(bytes) + " bytes)");
        return MRPT_ERR_OOM;
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    return MRPT_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int Scratch::ensure(size_t need, const char *what) {
    if (need <= bytes && ptr != nullptr) return MRPT_OK;
    release();
    size_t cap = need < 4096 ? 4096 : need + need / 4;
    int rc = dev_alloc(&ptr, cap, what);
    if (rc) return rc;
    bytes = cap;
    return MRPT_OK;
}

void Scratch::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

// The routing kernel reads the nonzeros of R as (dimension, value bits)
// pairs, two per 16-byte load: every column starts at an even pair index (a
// column of odd length leaves one unused pair after it), and rcol[c] holds
// (first pair, count) of column c.  The arithmetic order is unchanged.
static int upload_route_pairs(mrpt_index *idx) {
    const int64_t ncols = int64_t(idx->h_col_off.size()) - 1;
    std::vector<int2> rcol(size_t(ncols > 0 ? ncols : 0));
    int64_t total = 0;
    for (int64_t c = 0; c < ncols; ++c) {
        const int32_t cnt = idx->h_col_off[size_t(c) + 1] - idx->h_col_off[size_t(c)];
        rcol[size_t(c)] = make_int2(int32_t(total), cnt);
        total += (cnt + 1) & ~1;
    }
    const size_t bytes = size_t(total > 0 ? total : 2) * sizeof(int2);
    const size_t cbytes = size_t(ncols > 0 ? ncols : 1) * sizeof(int2);
    int rc = dev_alloc((void **)&idx->dv, bytes, "R routing pairs");
    if (!rc) rc = dev_alloc((void **)&idx->rcol, cbytes, "R routing columns");
    if (rc) return rc;
    idx->device_bytes += int64_t(bytes + cbytes);
    std::vector<int2> h(bytes / sizeof(int2), make_int2(0, 0));
    for (int64_t c = 0; c < ncols; ++c) {
        const int32_t e0 = idx->h_col_off[size_t(c)];
        for (int32_t k = 0; k < rcol[size_t(c)].y; ++k) {
            int32_t bits;
            memcpy(&bits, &idx->h_val[size_t(e0 + k)], sizeof(bits));
            h[size_t(rcol[size_t(c)].x + k)] = make_int2(idx->h_dim[size_t(e0 + k)], bits);
        }
    }
    cudaError_t e = cudaMemcpy(idx->dv, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ncols > 0)
        e = cudaMemcpy(idx->rcol, rcol.data(), cbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading R routing pairs");
    return MRPT_OK;
}

static void free_index(mrpt_index *idx) {
    if (!idx) return;
    cudaFree(idx->X);
    cudaFree(idx->col_off);
    cudaFree(idx->dim);
    cudaFree(idx->val);
    cudaFree(idx->dv);
    cudaFree(idx->rcol);
    cudaFree(idx->split);
    cudaFree(idx->leaf_off);
    cudaFree(idx->leaf_ids);
    cudaFree(idx->leaf4);
    cudaFree(idx->leaf_off4);
    cudaFree(idx->chunk_bnd);
    cudaFree(idx->Xb);
    cudaFree(idx->X8);
    cudaFree(idx->status);
    for (cudaEvent_t &ev : idx->ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t &ev : idx->pev)
        if (ev) cudaEventDestroy(ev);
    if (idx->copy_stream) cudaStreamDestroy(idx->copy_stream);
    idx->q_leaf.release();
    idx->q_stage.release();
    idx->o_stage.release();
    idx->dbg_stage.release();
    idx->q_cand.release();
    idx->shard.release();
    delete idx;
}

// Scratch of the two-kernel query path for m queries: candidate lists,
// work items, per-chunk partial top-k lists, |S| and per-query completion
// counters, each starting on a 256-byte boundary.
struct CandLayout {
    int32_t capq, chunk, max_items_q, ring;
    size_t lb, ib, pb, nb, total;
};

static CandLayout cand_layout(const mrpt_index *idx, int64_t m, int32_t k, int32_t v,
                              int32_t n_trees, int32_t precision, int32_t margin,
                              const mrpt_query_opts *opts) {
    CandLayout L{};
    const int64_t ks = int64_t(k) + margin;  // list length kept per chunk
    // |S| <= T ceil(n / 2^l) / v (Sec. III-B: every member of S holds at
    // least v of the T ceil(n / 2^l) votes), and |S| <= n: a list of that
    // length holds every candidate of any query
    const int64_t leaf_max = (idx->n + idx->L - 1) / idx->L;
    int64_t bound = int64_t(n_trees) * leaf_max / v;
    if (bound > idx->n) bound = idx->n;
    L.capq = int32_t(bound < 1 ? 1 : bound);
    // candidate-search work items: chunks of a list, at least 2(k + margin)
    // candidates and 64 (float32) or 32 (bfloat16) each, at most
    // CAND_ITEMS_MAX per query
    L.chunk = int32_t(std::max<int64_t>(precision != MRPT_PREC_FP32 ? 32 : 64, ((2 * ks + 31) / 32) * 32));
    if (opts && opts->chunk > 0) L.chunk = int32_t(std::max<int64_t>(opts->chunk, ks));
    L.ring = (opts && opts->ring > 0) ? std::min<int32_t>(std::max<int32_t>(opts->ring, 2), 16) : 0;
    L.max_items_q = int32_t(std::min<int64_t>((int64_t(L.capq) + L.chunk - 1) / L.chunk, CAND_ITEMS_MAX));
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    L.lb = up(size_t(m) * size_t(L.capq) * 4);
    L.ib = up(size_t(m) * size_t(L.max_items_q) * 8);
    L.pb = up(size_t(m) * size_t(L.max_items_q) * size_t(ks) * 4);
    L.nb = up(size_t(m) * 4);
    L.total = L.lb + L.ib + 2 * L.pb + 2 * L.nb;
    return L;
}

static void cand_carve(const CandLayout &L, char *base, int64_t m, QueryLaunch &ql) {
    (void)m;
    ql.capq = L.capq;
    ql.chunk = L.chunk;
    ql.max_items_q = L.max_items_q;
    ql.ring = L.ring;
    ql.cand_list = reinterpret_cast<int32_t *>(base);
    ql.items = reinterpret_cast<int2 *>(base + L.lb);
    ql.part_d = reinterpret_cast<float *>(base + L.lb + L.ib);
    ql.part_i = reinterpret_cast<int32_t *>(base + L.lb + L.ib + L.pb);
    ql.ncand = reinterpret_cast<int32_t *>(base + L.lb + L.ib + 2 * L.pb);
    ql.done = reinterpret_cast<int32_t *>(base + L.lb + L.ib + 2 * L.pb + L.nb);
}

}  // namespace mrpt

// A captured query graph and everything it reads or writes.
struct mrpt_plan {
    mrpt_index *idx = nullptr;
    int64_t m_max = 0;
    int32_t k = 0, v = 0, n_trees = 0;
    mrpt::Scratch buf;          // record, counters, staging, query scratch
    mrpt::QueryRecord *rec = nullptr;
    uint32_t *counters = nullptr;
    float *q_stage = nullptr;
    int32_t *ids_stage = nullptr;
    float *dists_stage = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace mrpt;

extern "C" {

const char *mrpt_last_error(void) { return g_last_error.c_str(); }

int mrpt_debug_fail_alloc_after(int32_t after) {
    g_fail_after.store(after < 0 ? -1 : after);
    return MRPT_OK;
}

int mrpt_debug_row_wait_tries(int32_t tries) {
    g_row_wait_tries.store(tries < 0 ? -1 : tries);
    return MRPT_OK;
}

int mrpt_build(const float *data, int64_t n, int32_t d, int32_t T, int32_t l, float density,
               uint64_t seed, mrpt_index **out) {
    return mrpt_build_ex(data, n, d, T, l, density, seed, nullptr, out);
}

int mrpt_build_ex(const float *data, int64_t n, int32_t d, int32_t T, int32_t l, float density,
                  uint64_t seed, const mrpt_build_opts *opts, mrpt_index **out) {
    clear_error();
    if (!out) {
        set_error("mrpt_build: out is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t sparsity = opts ? opts->sparsity : MRPT_SPARSITY_BERNOULLI;
    if (sparsity != MRPT_SPARSITY_BERNOULLI && sparsity != MRPT_SPARSITY_FIXED) {
        set_error("mrpt_build: unknown sparsity " + std::to_string(sparsity));
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t tree_offset = opts ? opts->tree_offset : 0;
    if (tree_offset < 0 || int64_t(tree_offset) + T > MRPT_MAX_TREES) {
        set_error("mrpt_build: need 0 <= tree_offset and tree_offset + T <= " + std::to_string(MRPT_MAX_TREES));
        return MRPT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!data || n < 1 || n > int64_t(INT32_MAX) || d < 1 || d > MRPT_MAX_DIM || T < 1 ||
        T > MRPT_MAX_TREES || l < 0 || l > MRPT_MAX_DEPTH || (int64_t(1) << l) > n ||
        !(density <= 1.0f) || std::isnan(density)) {
        set_error("mrpt_build: invalid argument (need data != NULL, 1 <= n < 2^31, 1 <= d <= " +
                  std::to_string(MRPT_MAX_DIM) + ", 1 <= T <= " + std::to_string(MRPT_MAX_TREES) +
                  ", 0 <= l <= " + std::to_string(MRPT_MAX_DEPTH) +
                  ", 2^l <= n, density <= 1)");
        return MRPT_ERR_INVALID_ARG;
    }
    if (density <= 0.0f) density = float(1.0 / std::sqrt(double(d)));

    mrpt_index *idx = new (std::nothrow) mrpt_index();
    if (!idx) {
        set_error("mrpt_build: host allocation failed");
        return MRPT_ERR_OOM;
    }
    int rc = MRPT_OK;
    cudaGetDevice(&idx->device);
    idx->n = n;
    idx->d = d;
    idx->dpad = (d + 7) & ~7;
    idx->T = T;
    idx->l = l;
    idx->L = int64_t(1) << l;
    idx->density = density;
    idx->seed = seed;
    idx->tree_offset = tree_offset;
    idx->stream = nullptr;
    cudaStream_t s = idx->stream;

    auto fail = [&](int code) {
        free_index(idx);
        return code;
    };

    // ---- data: n x dpad, zero padded
    const size_t xbytes = size_t(n) * size_t(idx->dpad) * sizeof(float);
    if ((rc = dev_alloc((void **)&idx->X, xbytes, "index data"))) return fail(rc);
    idx->device_bytes += int64_t(xbytes);
    {
        cudaError_t e = cudaMemsetAsync(idx->X, 0, xbytes, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(idx->X, size_t(idx->dpad) * sizeof(float), data,
                                  size_t(d) * sizeof(float), size_t(d) * sizeof(float), size_t(n),
                                  cudaMemcpyDefault, s);
        if (e != cudaSuccess) return fail(cuda_fail(e, "mrpt_build: copying data"));
    }
    bool nonfinite = false;
    if ((rc = check_finite(idx->X, n, idx->dpad, d, s, &nonfinite))) return fail(rc);
    if (nonfinite) {
        set_error("mrpt_build: data holds NaN or Inf");
        return fail(MRPT_ERR_NONFINITE_INPUT);
    }

    // ---- random matrix (Algorithm 1, Sec. II-B/II-C)
    generate_random_matrix(T, l, d, density, seed, sparsity, tree_offset, idx->h_col_off, idx->h_dim,
                           idx->h_val);
    idx->nnz = int64_t(idx->h_dim.size());
    const size_t cbytes = idx->h_col_off.size() * sizeof(int32_t);
    const size_t nbytes = size_t(idx->nnz) * sizeof(int32_t);
    if ((rc = dev_alloc((void **)&idx->col_off, cbytes, "R column offsets"))) return fail(rc);
    if ((rc = dev_alloc((void **)&idx->dim, nbytes, "R dimensions"))) return fail(rc);
    if ((rc = dev_alloc((void **)&idx->val, nbytes, "R values"))) return fail(rc);
    idx->device_bytes += int64_t(cbytes + 2 * nbytes);
    {
        cudaError_t e = cudaMemcpy(idx->col_off, idx->h_col_off.data(), cbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nbytes)
            e = cudaMemcpy(idx->dim, idx->h_dim.data(), nbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && nbytes)
            e = cudaMemcpy(idx->val, idx->h_val.data(), nbytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "mrpt_build: uploading R"));
    }
    if ((rc = upload_route_pairs(idx))) return fail(rc);

    // ---- trees (Algorithm 2)
    const size_t sbytes = size_t(T) * size_t(idx->L - 1) * sizeof(float);
    if ((rc = dev_alloc((void **)&idx->split, sbytes, "split values"))) return fail(rc);
    if ((rc = dev_alloc((void **)&idx->leaf_off, size_t(idx->L + 1) * sizeof(int32_t), "leaf offsets")))
        return fail(rc);
    if ((rc = dev_alloc((void **)&idx->status, 8 * sizeof(uint32_t), "status words"))) return fail(rc);
    idx->device_bytes += int64_t(sbytes + size_t(idx->L + 1) * 4 + 32);
    {
        cudaError_t e = cudaMemset(idx->status, 0, 8 * sizeof(uint32_t));
        if (e != cudaSuccess) return fail(cuda_fail(e, "mrpt_build: status"));
    }
    if ((rc = grow_trees_device(idx))) return fail(rc);
    if ((rc = build_vote_layout(idx))) return fail(rc);
    *out = idx;
    return MRPT_OK;
}

int mrpt_free(mrpt_index *idx) {
    clear_error();
    if (idx) {
        cudaStreamSynchronize(idx->stream);
        free_index(idx);
    }
    return MRPT_OK;
}

int mrpt_set_stream(mrpt_index *idx, void *stream) {
    clear_error();
    if (!idx) {
        set_error("mrpt_set_stream: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    idx->stream = static_cast<cudaStream_t>(stream);
    return MRPT_OK;
}

int mrpt_sync(mrpt_index *idx) {
    clear_error();
    if (!idx) {
        set_error("mrpt_sync: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    uint32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, idx->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, idx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
    if (e == cudaSuccess && st) e = cudaMemsetAsync(idx->status, 0, sizeof(uint32_t), idx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mrpt_sync");
    if (st & STATUS_TIMEOUT) {
        set_error("a bounded device wait ran out");
        return MRPT_ERR_TIMEOUT;
    }
    if (st & STATUS_NONFINITE_QUERY) {
        set_error("a query held NaN or Inf");
        return MRPT_ERR_NONFINITE_INPUT;
    }
    return MRPT_OK;
}

int mrpt_info(const mrpt_index *idx, mrpt_index_info *info) {
    clear_error();
    if (!idx || !info) {
        set_error("mrpt_info: NULL argument");
        return MRPT_ERR_INVALID_ARG;
    }
    info->n = idx->n;
    info->d = idx->d;
    info->T = idx->T;
    info->l = idx->l;
    info->density = idx->density;
    info->seed = idx->seed;
    info->nnz = idx->nnz;
    info->tree_offset = idx->tree_offset;
    info->device_bytes = idx->device_bytes + int64_t(idx->q_leaf.bytes + idx->q_stage.bytes +
                                                     idx->o_stage.bytes + idx->dbg_stage.bytes +
                                                     idx->q_cand.bytes + idx->shard.bytes);
    return MRPT_OK;
}

// A vote-table choice the index can take (mrpt_query_opts.vote_table).
static bool vote_table_ok(const mrpt_index *idx, int32_t n_trees, int32_t vt) {
    if (vt == 0 || vt == MRPT_VOTE_COUNTERS) return true;
    if (vt != MRPT_VOTE_HASH) return false;
    const int64_t leaf_max = (idx->n + idx->L - 1) / idx->L;
    return int64_t(n_trees) * leaf_max <= MRPT_VOTE_HASH_ENTRIES && idx->n < (int64_t(1) << 24);
}

// Host queries in batches of at least this many are copied in chunks, each
// chunk routed as soon as it has arrived, so the copy overlaps routing.
constexpr int kPipeChunks = 4;
constexpr int64_t kPipeMinQueries = 8192;

int mrpt_query_ex(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
                  const mrpt_query_opts *opts, int32_t *out_ids, float *out_dists) {
    clear_error();
    if (!idx) {
        set_error("mrpt_query: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t n_trees = (opts && opts->n_trees > 0) ? opts->n_trees : idx->T;
    if (m < 0 || (m > 0 && (!Q || !out_ids || !out_dists)) || k < 1 || k > MRPT_MAX_K || v < 1 ||
        n_trees > idx->T || v > n_trees) {
        set_error("mrpt_query: invalid argument (need m >= 0, non-NULL buffers, 1 <= k <= " +
                  std::to_string(MRPT_MAX_K) + ", 1 <= v <= n_trees <= T)");
        return MRPT_ERR_INVALID_ARG;
    }
    if (opts && (opts->chunk < 0 || opts->ring < 0)) {
        set_error("mrpt_query: chunk and ring must be >= 0");
        return MRPT_ERR_INVALID_ARG;
    }
    if (opts && !vote_table_ok(idx, n_trees, opts->vote_table)) {
        set_error("mrpt_query: vote_table must be 0, 1 or 2, and 2 needs n_trees * ceil(n / 2^l) <= " +
                  std::to_string(MRPT_VOTE_HASH_ENTRIES) + " and n < 2^24");
        return MRPT_ERR_INVALID_ARG;
    }
    if (opts && opts->cand && opts->cand_cap < 0) {
        set_error("mrpt_query: cand_cap < 0");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t precision = opts ? opts->precision : MRPT_PREC_FP32;
    const int32_t margin = (opts && precision != MRPT_PREC_FP32) ? opts->margin : 0;
    if (precision != MRPT_PREC_FP32 && precision != MRPT_PREC_BF16 && precision != MRPT_PREC_FP8) {
        set_error("mrpt_query: unknown precision");
        return MRPT_ERR_INVALID_ARG;
    }
    if (precision != MRPT_PREC_FP32) {
        if ((precision == MRPT_PREC_BF16 && !idx->Xb) || (precision == MRPT_PREC_FP8 && !idx->X8)) {
            set_error("mrpt_query: reduced-precision distances need mrpt_add_lowp(idx, precision) first");
            return MRPT_ERR_INVALID_ARG;
        }
        if (opts->path != 0 || margin < 0 || k + margin > MRPT_MAX_K) {
            set_error("mrpt_query: reduced-precision distances need path 0 and 0 <= margin, k + margin <= " +
                      std::to_string(MRPT_MAX_K));
            return MRPT_ERR_INVALID_ARG;
        }
    }
    if (m == 0) return MRPT_OK;
    cudaStream_t s = idx->stream;
    int rc;
    bool any_host = false;

    // ---- inputs
    const float *Qd = Q;
    const bool q_host = !is_device_ptr(Q);
    const bool chunked_in = q_host && m >= kPipeMinQueries &&
                            (!opts || (!opts->proj && !opts->leaf && !opts->stage_ms));
    if (q_host) {
        any_host = true;
        const size_t qb = size_t(m) * size_t(idx->d) * sizeof(float);
        if ((rc = idx->q_stage.ensure(qb, "query staging"))) return rc;
        if (!chunked_in) MRPT_CUDA_TRY(cudaMemcpyAsync(idx->q_stage.ptr, Q, qb, cudaMemcpyHostToDevice, s));
        Qd = static_cast<const float *>(idx->q_stage.ptr);
    }
    // ---- outputs (device buffers in place, host buffers staged)
    const bool ids_dev = is_device_ptr(out_ids);
    const bool dists_dev = is_device_ptr(out_dists);
    const size_t ob = size_t(m) * size_t(k) * 4;
    if (!ids_dev || !dists_dev) {
        any_host = true;
        if ((rc = idx->o_stage.ensure(2 * ob, "output staging"))) return rc;
    }
    int32_t *ids_d = ids_dev ? out_ids : static_cast<int32_t *>(idx->o_stage.ptr);
    float *dists_d = dists_dev ? out_dists
                               : reinterpret_cast<float *>(static_cast<char *>(idx->o_stage.ptr) + ob);

    // ---- debug outputs (staged when on the host)
    QueryLaunch ql{};
    ql.Q = Qd;
    ql.m = m;
    ql.k = k;
    ql.v = v;
    ql.n_trees = n_trees;
    ql.out_ids = ids_d;
    ql.out_dists = dists_d;
    const size_t leaf_b = size_t(m) * size_t(n_trees) * 4;
    struct Dbg {
        void *user;
        size_t bytes;
        size_t off;
    } dbg[5] = {};
    size_t dbg_total = 0;
    if (opts) {
        void *ptrs[5] = {opts->proj, opts->leaf, opts->votes, opts->n_cand, opts->cand};
        size_t sizes[5] = {size_t(m) * size_t(n_trees) * size_t(idx->l) * 4, leaf_b,
                           size_t(m) * size_t(idx->n), size_t(m) * 8,
                           size_t(m) * size_t(opts->cand_cap) * 4};
        for (int i = 0; i < 5; ++i) {
            dbg[i].user = ptrs[i];
            dbg[i].bytes = sizes[i];
            if (ptrs[i] && !is_device_ptr(ptrs[i])) {
                dbg[i].off = dbg_total;
                dbg_total += (sizes[i] + 255) & ~size_t(255);
                any_host = true;
            } else {
                dbg[i].off = SIZE_MAX;
            }
        }
        if (dbg_total && (rc = idx->dbg_stage.ensure(dbg_total, "debug staging"))) return rc;
        auto dev_of = [&](int i) -> void * {
            if (!dbg[i].user) return nullptr;
            if (dbg[i].off == SIZE_MAX) return dbg[i].user;
            return static_cast<char *>(idx->dbg_stage.ptr) + dbg[i].off;
        };
        ql.proj = static_cast<float *>(dev_of(0));
        ql.leaf = static_cast<int32_t *>(dev_of(1));
        ql.votes = static_cast<uint8_t *>(dev_of(2));
        ql.n_cand = static_cast<int64_t *>(dev_of(3));
        ql.cand = static_cast<int32_t *>(dev_of(4));
        ql.cand_cap = opts->cand_cap;
        ql.stage_ms = opts->stage_ms;
    }
    if (!ql.leaf) {
        if ((rc = idx->q_leaf.ensure(leaf_b, "leaf-of-query scratch"))) return rc;
        ql.leaf = static_cast<int32_t *>(idx->q_leaf.ptr);
    }
    ql.path = opts ? opts->path : 0;
    ql.precision = precision;
    ql.margin = margin;
    ql.vote_table = opts ? opts->vote_table : 0;
    // two-kernel path: candidate lists for mb queries at a time, mb = m
    // unless their scratch would pass kCandScratchBudget
    int64_t mb = m;
    if (ql.path == 0) {
        CandLayout lay = cand_layout(idx, m, k, v, n_trees, precision, margin, opts);
        if (lay.total > kCandScratchBudget) {
            const CandLayout one = cand_layout(idx, 1, k, v, n_trees, precision, margin, opts);
            mb = std::max<int64_t>(1, int64_t(kCandScratchBudget / one.total));
            lay = cand_layout(idx, mb, k, v, n_trees, precision, margin, opts);
        }
        if ((rc = idx->q_cand.ensure(lay.total, "candidate lists"))) return rc;
        cand_carve(lay, static_cast<char *>(idx->q_cand.ptr), mb, ql);
    }

    if (chunked_in) {
        // copy the queries in chunks on a second stream; route each chunk
        // on the index's stream as soon as it has arrived
        if (!idx->copy_stream) MRPT_CUDA_TRY(cudaStreamCreateWithFlags(&idx->copy_stream, cudaStreamNonBlocking));
        for (cudaEvent_t &e : idx->pev)
            if (!e) MRPT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaStream_t cs = idx->copy_stream;
        MRPT_CUDA_TRY(cudaEventRecord(idx->pev[0], s));  // after work already queued
        MRPT_CUDA_TRY(cudaStreamWaitEvent(cs, idx->pev[0], 0));
        const int64_t mc = (m + kPipeChunks - 1) / kPipeChunks;
        const size_t row = size_t(idx->d) * sizeof(float);
        int c = 0;
        for (int64_t q0 = 0; q0 < m; q0 += mc, ++c) {
            const int64_t mq = std::min(mc, m - q0);
            char *dst = static_cast<char *>(idx->q_stage.ptr) + size_t(q0) * row;
            MRPT_CUDA_TRY(cudaMemcpyAsync(dst, reinterpret_cast<const char *>(Q) + size_t(q0) * row,
                                          size_t(mq) * row, cudaMemcpyHostToDevice, cs));
            MRPT_CUDA_TRY(cudaEventRecord(idx->pev[1 + c], cs));
            MRPT_CUDA_TRY(cudaStreamWaitEvent(s, idx->pev[1 + c], 0));
            QueryLaunch qc = ql;
            qc.Q = reinterpret_cast<const float *>(dst);
            qc.m = mq;
            qc.leaf = ql.leaf + q0 * n_trees;
            if ((rc = launch_route_only(idx, qc))) return rc;
        }
        ql.routed = true;
    }
    if (mb >= m) {
        if ((rc = launch_query(idx, ql))) return rc;
    } else {
        // consecutive sub-batches reuse the candidate scratch; stage times add up
        float acc[4] = {0.f, 0.f, 0.f, 0.f}, part[4];
        for (int64_t q0 = 0; q0 < m; q0 += mb) {
            QueryLaunch qb = ql;
            qb.m = std::min(mb, m - q0);
            qb.Q = ql.Q + q0 * idx->d;
            qb.out_ids = ql.out_ids + q0 * k;
            qb.out_dists = ql.out_dists + q0 * k;
            qb.leaf = ql.leaf + q0 * n_trees;
            if (ql.proj) qb.proj = ql.proj + q0 * int64_t(n_trees) * idx->l;
            if (ql.votes) qb.votes = ql.votes + q0 * idx->n;
            if (ql.n_cand) qb.n_cand = ql.n_cand + q0;
            if (ql.cand) qb.cand = ql.cand + q0 * ql.cand_cap;
            qb.stage_ms = ql.stage_ms ? part : nullptr;
            if ((rc = launch_query(idx, qb))) return rc;
            if (ql.stage_ms)
                for (int i = 0; i < 4; ++i) acc[i] += part[i];
        }
        if (ql.stage_ms)
            for (int i = 0; i < 4; ++i) ql.stage_ms[i] = acc[i];
    }

    // ---- copy staged results back
    if (!ids_dev) MRPT_CUDA_TRY(cudaMemcpyAsync(out_ids, ids_d, ob, cudaMemcpyDeviceToHost, s));
    if (!dists_dev) MRPT_CUDA_TRY(cudaMemcpyAsync(out_dists, dists_d, ob, cudaMemcpyDeviceToHost, s));
    for (int i = 0; i < 5; ++i)
        if (dbg[i].user && dbg[i].off != SIZE_MAX)
            MRPT_CUDA_TRY(cudaMemcpyAsync(dbg[i].user, static_cast<char *>(idx->dbg_stage.ptr) + dbg[i].off,
                                          dbg[i].bytes, cudaMemcpyDeviceToHost, s));
    if (any_host) return mrpt_sync(idx);
    return MRPT_OK;
}

int mrpt_add_lowp(mrpt_index *idx, int32_t precision) {
    clear_error();
    if (!idx || (precision != MRPT_PREC_BF16 && precision != MRPT_PREC_FP8)) {
        set_error("mrpt_add_lowp: need an index and precision MRPT_PREC_BF16 or MRPT_PREC_FP8");
        return MRPT_ERR_INVALID_ARG;
    }
    return precision == MRPT_PREC_BF16 ? make_bf16_copy(idx) : make_fp8_copy(idx);
}

int mrpt_query(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v, int32_t *out_ids,
               float *out_dists) {
    return mrpt_query_ex(idx, Q, m, k, v, nullptr, out_ids, out_dists);
}

int mrpt_plan_free(mrpt_plan *plan) {
    clear_error();
    if (!plan) return MRPT_OK;
    if (plan->idx) cudaStreamSynchronize(plan->idx->stream);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    plan->buf.release();
    delete plan;
    return MRPT_OK;
}

int mrpt_plan_create(mrpt_index *idx, int64_t m_max, int32_t k, int32_t v,
                     const mrpt_query_opts *opts, mrpt_plan **out) {
    clear_error();
    if (!out || !idx) {
        set_error("mrpt_plan_create: NULL argument");
        return MRPT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const int32_t n_trees = (opts && opts->n_trees > 0) ? opts->n_trees : idx->T;
    const int32_t path = opts ? opts->path : 0;
    const int32_t precision = opts ? opts->precision : MRPT_PREC_FP32;
    const int32_t margin = (opts && precision != MRPT_PREC_FP32) ? opts->margin : 0;
    if (m_max < 1 || k < 1 || k > MRPT_MAX_K || v < 1 || n_trees > idx->T || v > n_trees ||
        (path != 0 && path != 1) ||
        (precision != MRPT_PREC_FP32 && precision != MRPT_PREC_BF16 && precision != MRPT_PREC_FP8) ||
        (precision == MRPT_PREC_BF16 && !idx->Xb) || (precision == MRPT_PREC_FP8 && !idx->X8) ||
        (precision != MRPT_PREC_FP32 && (path != 0 || margin < 0 || k + margin > MRPT_MAX_K)) ||
        (opts && (opts->chunk < 0 || opts->ring < 0 || opts->proj || opts->leaf || opts->votes ||
                  opts->n_cand || opts->cand || opts->stage_ms)) ||
        (opts && !vote_table_ok(idx, n_trees, opts->vote_table))) {
        set_error("mrpt_plan_create: invalid argument (need m_max >= 1, 1 <= k <= " +
                  std::to_string(MRPT_MAX_K) +
                  ", 1 <= v <= n_trees <= T, a valid path/precision, no debug outputs)");
        return MRPT_ERR_INVALID_ARG;
    }
    mrpt_plan *plan = new (std::nothrow) mrpt_plan();
    if (!plan) {
        set_error("mrpt_plan_create: host allocation failed");
        return MRPT_ERR_OOM;
    }
    plan->idx = idx;
    plan->m_max = m_max;
    plan->k = k;
    plan->v = v;
    plan->n_trees = n_trees;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t rec_b = 256, ctr_b = 256;
    const size_t q_b = up(size_t(m_max) * size_t(idx->d) * 4);
    const size_t o_b = up(size_t(m_max) * size_t(k) * 4);
    const size_t leaf_b = up(size_t(m_max) * size_t(n_trees) * 4);
    CandLayout lay{};
    if (path == 0) lay = cand_layout(idx, m_max, k, v, n_trees, precision, margin, opts);
    int rc = plan->buf.ensure(rec_b + ctr_b + q_b + 2 * o_b + leaf_b + lay.total, "query plan");
    if (rc) {
        delete plan;
        return rc;
    }
    char *base = static_cast<char *>(plan->buf.ptr);
    plan->rec = reinterpret_cast<QueryRecord *>(base);
    plan->counters = reinterpret_cast<uint32_t *>(base + rec_b);
    plan->q_stage = reinterpret_cast<float *>(base + rec_b + ctr_b);
    plan->ids_stage = reinterpret_cast<int32_t *>(base + rec_b + ctr_b + q_b);
    plan->dists_stage = reinterpret_cast<float *>(base + rec_b + ctr_b + q_b + o_b);
    int32_t *leaf = reinterpret_cast<int32_t *>(base + rec_b + ctr_b + q_b + 2 * o_b);
    char *cand_base = base + rec_b + ctr_b + q_b + 2 * o_b + leaf_b;

    QueryLaunch ql{};
    ql.Q = plan->q_stage;
    ql.m = m_max;
    ql.k = k;
    ql.v = v;
    ql.n_trees = n_trees;
    ql.out_ids = plan->ids_stage;
    ql.out_dists = plan->dists_stage;
    ql.leaf = leaf;
    ql.path = path;
    ql.precision = precision;
    ql.margin = margin;
    ql.vote_table = opts ? opts->vote_table : 0;
    if (path == 0) cand_carve(lay, cand_base, m_max, ql);
    ql.counters = plan->counters;
    ql.rec = plan->rec;
    ql.use_stream = true;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->counters, 0, ctr_b, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        mrpt_plan_free(plan);
        return cuda_fail(e, "mrpt_plan_create: stream");
    }
    ql.stream = cs;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = launch_query(idx, ql);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        plan->graph = g;
        if (rc == MRPT_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "mrpt_plan_create: capture");
    } else {
        rc = cuda_fail(e, "mrpt_plan_create: begin capture");
    }
    if (rc == MRPT_OK) {
        e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "mrpt_plan_create: instantiate");
    }
    cudaStreamDestroy(cs);
    if (rc != MRPT_OK) {
        mrpt_plan_free(plan);
        return rc;
    }
    *out = plan;
    return MRPT_OK;
}

int mrpt_plan_run(mrpt_plan *plan, const float *Q, int64_t m, int32_t *out_ids, float *out_dists) {
    clear_error();
    if (!plan) {
        set_error("mrpt_plan_run: plan is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    if (m < 0 || m > plan->m_max || (m > 0 && (!Q || !out_ids || !out_dists))) {
        set_error("mrpt_plan_run: need 0 <= m <= m_max and non-NULL buffers");
        return MRPT_ERR_INVALID_ARG;
    }
    if (m == 0) return MRPT_OK;
    mrpt_index *idx = plan->idx;
    cudaStream_t s = idx->stream;
    const size_t qb = size_t(m) * size_t(idx->d) * 4;
    const size_t ob = size_t(m) * size_t(plan->k) * 4;
    bool any_host = false;
    QueryRecord r{};
    r.m = m;
    if (is_device_ptr(Q)) {
        r.Q = Q;
    } else {
        any_host = true;
        MRPT_CUDA_TRY(cudaMemcpyAsync(plan->q_stage, Q, qb, cudaMemcpyHostToDevice, s));
        r.Q = plan->q_stage;
    }
    const bool ids_dev = is_device_ptr(out_ids), dists_dev = is_device_ptr(out_dists);
    any_host = any_host || !ids_dev || !dists_dev;
    r.out_ids = ids_dev ? out_ids : plan->ids_stage;
    r.out_dists = dists_dev ? out_dists : plan->dists_stage;
    int rc = set_record(plan->rec, r, s);
    if (rc) return rc;
    MRPT_CUDA_TRY(cudaGraphLaunch(plan->exec, s));
    if (!ids_dev) MRPT_CUDA_TRY(cudaMemcpyAsync(out_ids, plan->ids_stage, ob, cudaMemcpyDeviceToHost, s));
    if (!dists_dev) MRPT_CUDA_TRY(cudaMemcpyAsync(out_dists, plan->dists_stage, ob, cudaMemcpyDeviceToHost, s));
    if (any_host) return mrpt_sync(idx);
    return MRPT_OK;
}

// ---- save / load: "MRPTIDX1", header, R (compressed columns), split
// values, leaf lists, data.  Little-endian, as the host writes it.
namespace {
struct FileHeader {
    char magic[8];
    int64_t n;
    int32_t d, T, l;
    float density;
    uint64_t seed;
    int64_t nnz;
    int32_t tree_offset, reserved;
};

int write_all(FILE *f, const void *p, size_t bytes) { return fwrite(p, 1, bytes, f) == bytes ? 0 : -1; }
int read_all(FILE *f, void *p, size_t bytes) { return fread(p, 1, bytes, f) == bytes ? 0 : -1; }
}  // namespace

int mrpt_save(const mrpt_index *idx, const char *path) {
    clear_error();
    if (!idx || !path) {
        set_error("mrpt_save: NULL argument");
        return MRPT_ERR_INVALID_ARG;
    }
    MRPT_CUDA_TRY(cudaStreamSynchronize(idx->stream));
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error(std::string("mrpt_save: cannot open ") + path);
        return MRPT_ERR_INVALID_ARG;
    }
    FileHeader h{};
    memcpy(h.magic, "MRPTIDX2", 8);
    h.n = idx->n;
    h.d = idx->d;
    h.T = idx->T;
    h.l = idx->l;
    h.density = idx->density;
    h.seed = idx->seed;
    h.nnz = idx->nnz;
    h.tree_offset = idx->tree_offset;
    const size_t sb = size_t(idx->T) * size_t(idx->L - 1) * 4;
    const size_t ib = size_t(idx->T) * size_t(idx->n) * 4;
    const size_t xb = size_t(idx->n) * size_t(idx->d) * 4;
    std::string err;
    void *host = malloc(std::max(std::max(sb, ib), std::max(xb, size_t(1))));
    int bad = host ? 0 : -1;
    if (!bad) bad = write_all(f, &h, sizeof(h));
    if (!bad) bad = write_all(f, idx->h_col_off.data(), idx->h_col_off.size() * 4);
    if (!bad && idx->nnz) bad = write_all(f, idx->h_dim.data(), size_t(idx->nnz) * 4);
    if (!bad && idx->nnz) bad = write_all(f, idx->h_val.data(), size_t(idx->nnz) * 4);
    cudaError_t e = cudaSuccess;
    if (!bad && sb) {
        e = cudaMemcpy(host, idx->split, sb, cudaMemcpyDeviceToHost);
        bad = e != cudaSuccess ? -2 : write_all(f, host, sb);
    }
    if (!bad) {
        e = cudaMemcpy(host, idx->leaf_ids, ib, cudaMemcpyDeviceToHost);
        bad = e != cudaSuccess ? -2 : write_all(f, host, ib);
    }
    if (!bad) {
        e = cudaMemcpy2D(host, size_t(idx->d) * 4, idx->X, size_t(idx->dpad) * 4, size_t(idx->d) * 4,
                         size_t(idx->n), cudaMemcpyDeviceToHost);
        bad = e != cudaSuccess ? -2 : write_all(f, host, xb);
    }
    free(host);
    if (fclose(f) != 0 && !bad) bad = -1;
    if (bad == -2) return cuda_fail(e, "mrpt_save");
    if (bad) {
        set_error(host ? "mrpt_save: write failed" : "mrpt_save: host allocation failed");
        return host ? MRPT_ERR_INVALID_ARG : MRPT_ERR_OOM;
    }
    return MRPT_OK;
}

int mrpt_load(const char *path, mrpt_index **out) {
    clear_error();
    if (!path || !out) {
        set_error("mrpt_load: NULL argument");
        return MRPT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error(std::string("mrpt_load: cannot open ") + path);
        return MRPT_ERR_INVALID_ARG;
    }
    FileHeader h{};
    if (read_all(f, &h, sizeof(h)) || memcmp(h.magic, "MRPTIDX2", 8) != 0 || h.n < 1 || h.d < 1 ||
        h.d > MRPT_MAX_DIM || h.T < 1 || h.T > MRPT_MAX_TREES || h.l < 0 || h.l > MRPT_MAX_DEPTH ||
        (int64_t(1) << h.l) > h.n || h.nnz < 0 || h.tree_offset < 0 ||
        int64_t(h.tree_offset) + h.T > MRPT_MAX_TREES) {
        fclose(f);
        set_error("mrpt_load: not an index file or unsupported header");
        return MRPT_ERR_INVALID_ARG;
    }
    mrpt_index *idx = new (std::nothrow) mrpt_index();
    if (!idx) {
        fclose(f);
        set_error("mrpt_load: host allocation failed");
        return MRPT_ERR_OOM;
    }
    cudaGetDevice(&idx->device);
    idx->n = h.n;
    idx->d = h.d;
    idx->dpad = (h.d + 7) & ~7;
    idx->T = h.T;
    idx->l = h.l;
    idx->L = int64_t(1) << h.l;
    idx->density = h.density;
    idx->seed = h.seed;
    idx->nnz = h.nnz;
    idx->tree_offset = h.tree_offset;
    auto fail = [&](int code, const char *msg) {
        fclose(f);
        if (msg) set_error(msg);
        free_index(idx);
        return code;
    };
    idx->h_col_off.resize(size_t(h.T) * h.l + 1);
    idx->h_dim.resize(size_t(h.nnz));
    idx->h_val.resize(size_t(h.nnz));
    if (read_all(f, idx->h_col_off.data(), idx->h_col_off.size() * 4) ||
        (h.nnz && read_all(f, idx->h_dim.data(), size_t(h.nnz) * 4)) ||
        (h.nnz && read_all(f, idx->h_val.data(), size_t(h.nnz) * 4)) ||
        idx->h_col_off.back() != h.nnz)
        return fail(MRPT_ERR_INVALID_ARG, "mrpt_load: truncated or inconsistent random matrix");
    for (int32_t x : idx->h_dim)
        if (x < 0 || x >= h.d) return fail(MRPT_ERR_INVALID_ARG, "mrpt_load: dimension out of range");
    const size_t cb = idx->h_col_off.size() * 4, nb = size_t(h.nnz) * 4;
    const size_t sb = size_t(h.T) * size_t(idx->L - 1) * 4;
    const size_t ib = size_t(h.T) * size_t(h.n) * 4;
    const size_t xb = size_t(h.n) * size_t(h.d) * 4;
    int rc;
    if ((rc = dev_alloc((void **)&idx->col_off, cb, "R column offsets")) ||
        (rc = dev_alloc((void **)&idx->dim, nb, "R dimensions")) ||
        (rc = dev_alloc((void **)&idx->val, nb, "R values")) ||
        (rc = dev_alloc((void **)&idx->split, sb, "split values")) ||
        (rc = dev_alloc((void **)&idx->leaf_off, size_t(idx->L + 1) * 4, "leaf offsets")) ||
        (rc = dev_alloc((void **)&idx->leaf_ids, ib + 16, "leaf ids")) ||
        (rc = dev_alloc((void **)&idx->status, 8 * sizeof(uint32_t), "status words")) ||
        (rc = dev_alloc((void **)&idx->X, size_t(h.n) * size_t(idx->dpad) * 4, "index data")))
        return fail(rc, nullptr);
    idx->device_bytes = int64_t(cb + 2 * nb + sb + size_t(idx->L + 1) * 4 + ib + 32 +
                                size_t(h.n) * size_t(idx->dpad) * 4);
    void *host = malloc(std::max(std::max(sb, ib), std::max(xb, size_t(1))));
    if (!host) return fail(MRPT_ERR_OOM, "mrpt_load: host allocation failed");
    cudaError_t e = cudaMemset(idx->status, 0, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(idx->col_off, idx->h_col_off.data(), cb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nb) e = cudaMemcpy(idx->dim, idx->h_dim.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nb) e = cudaMemcpy(idx->val, idx->h_val.data(), nb, cudaMemcpyHostToDevice);
    bool short_read = false;
    if (e == cudaSuccess && sb) {
        short_read = read_all(f, host, sb) != 0;
        if (!short_read) e = cudaMemcpy(idx->split, host, sb, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !short_read) {
        short_read = read_all(f, host, ib) != 0;
        const int32_t *ids = static_cast<const int32_t *>(host);
        for (size_t i = 0; !short_read && i < size_t(h.T) * size_t(h.n); ++i)
            if (ids[i] < 0 || ids[i] >= h.n) short_read = true;
        if (!short_read) e = cudaMemcpy(idx->leaf_ids, host, ib, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !short_read) {
        short_read = read_all(f, host, xb) != 0;
        if (!short_read) e = cudaMemset(idx->X, 0, size_t(h.n) * size_t(idx->dpad) * 4);
        if (!short_read && e == cudaSuccess)
            e = cudaMemcpy2D(idx->X, size_t(idx->dpad) * 4, host, size_t(h.d) * 4, size_t(h.d) * 4,
                             size_t(h.n), cudaMemcpyHostToDevice);
    }
    free(host);
    if (e != cudaSuccess) {
        const int code = cuda_fail(e, "mrpt_load");
        fclose(f);
        free_index(idx);
        return code;
    }
    if (short_read) return fail(MRPT_ERR_INVALID_ARG, "mrpt_load: truncated file or leaf id out of range");
    fclose(f);
    if ((rc = compute_leaf_offsets(idx)) || (rc = upload_route_pairs(idx)) || (rc = build_vote_layout(idx))) {
        free_index(idx);
        return rc;
    }
    *out = idx;
    return MRPT_OK;
}

int64_t mrpt_export_size(const mrpt_index *idx, int32_t what) {
    clear_error();
    if (!idx) {
        set_error("mrpt_export_size: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    switch (what) {
        case MRPT_EXPORT_R_COL_OFF: return int64_t(idx->h_col_off.size()) * 4;
        case MRPT_EXPORT_R_DIM: return idx->nnz * 4;
        case MRPT_EXPORT_R_VAL: return idx->nnz * 4;
        case MRPT_EXPORT_SPLIT: return int64_t(idx->T) * (idx->L - 1) * 4;
        case MRPT_EXPORT_LEAF_OFF: return int64_t(idx->T) * (idx->L + 1) * 4;
        case MRPT_EXPORT_LEAF_IDS: return int64_t(idx->T) * idx->n * 4;
        case MRPT_EXPORT_DATA: return idx->n * int64_t(idx->d) * 4;
        default: break;
    }
    set_error("mrpt_export_size: unknown item");
    return MRPT_ERR_INVALID_ARG;
}

int mrpt_export(const mrpt_index *idx, int32_t what, void *dst, int64_t dst_bytes) {
    const int64_t need = mrpt_export_size(idx, what);
    if (need < 0) return int(need);
    if (!dst || dst_bytes < need) {
        set_error("mrpt_export: dst is NULL or too small");
        return MRPT_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaStreamSynchronize(idx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mrpt_export");
    switch (what) {
        case MRPT_EXPORT_R_COL_OFF:
            e = cudaMemcpy(dst, idx->h_col_off.data(), size_t(need), cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_R_DIM:
            if (need) e = cudaMemcpy(dst, idx->h_dim.data(), size_t(need), cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_R_VAL:
            if (need) e = cudaMemcpy(dst, idx->h_val.data(), size_t(need), cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_SPLIT:
            if (need) e = cudaMemcpy(dst, idx->split, size_t(need), cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_LEAF_OFF:
            for (int32_t t = 0; t < idx->T && e == cudaSuccess; ++t)
                e = cudaMemcpy(static_cast<char *>(dst) + size_t(t) * size_t(idx->L + 1) * 4,
                               idx->leaf_off, size_t(idx->L + 1) * 4, cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_LEAF_IDS:
            e = cudaMemcpy(dst, idx->leaf_ids, size_t(need), cudaMemcpyDefault);
            break;
        case MRPT_EXPORT_DATA:
            e = cudaMemcpy2D(dst, size_t(idx->d) * 4, idx->X, size_t(idx->dpad) * 4,
                             size_t(idx->d) * 4, size_t(idx->n), cudaMemcpyDefault);
            break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mrpt_export");
    return MRPT_OK;
}

}  // extern "C"
