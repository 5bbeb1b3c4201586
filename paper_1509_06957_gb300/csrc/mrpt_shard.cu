// Tree-sharded voting (Sec. I-C: the trees are independent, so they may be
// spread over machines).  A shard is an index built with a tree offset: it
// holds trees t0 .. t0+T-1 of the random source.  Each shard counts, per
// query, the votes of its own trees as a sparse (id, count) list
// (mrpt_vote_counts); after the lists of every shard have been exchanged,
// the owner of a query adds them up to F(x;q), keeps S = {x : F >= v}
// (Sec. III-A) and runs the exact search on S (mrpt_query_from_counts).
//
// Both steps go through dense vote rows in global memory (one 8-bit
// counter per point, 4 per word, updated by L2 atomics) for a batch of
// queries at a time, then one ordered pass per row that writes the ids
// whose count passes a threshold, ascending.  This is the exchange path,
// not the single-GPU hot path: it trades the shared-memory counters of the
// vote kernels for code that works the same for any n.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mrpt_internal.cuh"

namespace mrpt {
namespace {

constexpr int SH_THREADS = 256;
constexpr int SH_WARPS = SH_THREADS / 32;
// dense vote rows held at once (bytes)
constexpr size_t kDenseBudget = size_t(256) << 20;

// Row r (query q0 + r): every id x of the query's leaf in each of the
// n_trees trees adds one vote to byte x & 3 of word x >> 2.  A counter
// reaches at most n_trees <= 255, so no byte carries into its neighbour.
__global__ void k_dense_votes(const int32_t *__restrict__ leaf_of_q, int32_t n_trees,
                              const int32_t *__restrict__ leaf_off, const int32_t *__restrict__ leaf_ids,
                              int64_t n, int64_t mb, int64_t row_words, uint32_t *__restrict__ dense) {
    for (int64_t p = blockIdx.x; p < mb * n_trees; p += gridDim.x) {
        const int64_t r = p / n_trees;
        const int t = int(p - r * n_trees);
        const int32_t lf = leaf_of_q[r * n_trees + t];
        const int32_t b = leaf_off[lf], e = leaf_off[lf + 1];
        const int32_t *ids = leaf_ids + int64_t(t) * n;
        uint32_t *row = dense + r * row_words;
        for (int32_t i = b + int32_t(threadIdx.x); i < e; i += int32_t(blockDim.x)) {
            const int32_t x = ids[i];
            atomicAdd(row + (x >> 2), 1u << (8 * (x & 3)));
        }
    }
}

// Row r (query q0 + r) += the query's (id, count) pairs [off[q], off[q+1]).
// Ids outside [0, n) are skipped.  The counts of one id summed over the
// shards are at most the total number of trees (<= 255), so no byte
// carries into its neighbour.
__global__ void k_sparse_to_dense(const int64_t *__restrict__ off, const int32_t *__restrict__ ids,
                                  const uint8_t *__restrict__ counts, int64_t q0, int64_t mb, int64_t n,
                                  int64_t row_words, uint32_t *__restrict__ dense) {
    for (int64_t r = blockIdx.x; r < mb; r += gridDim.x) {
        const int64_t b = off[q0 + r], e = off[q0 + r + 1];
        uint32_t *row = dense + r * row_words;
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            const int32_t x = ids[i];
            if (x < 0 || x >= n) continue;
            atomicAdd(row + (x >> 2), uint32_t(counts[i]) << (8 * (x & 3)));
        }
    }
}

// Bit 7 of byte b of the result is set iff byte b of c is >= thr
// (1 <= thr <= 255): with add4 = (thr <= 128 ? 128 - thr : 256 - thr) per
// byte, (c & 0x7f) + add never carries out of its byte and its bit 7 says
// (c & 0x7f) >= thr - 128 (thr > 128) or >= thr (else; a byte >= 128 then
// passes whatever its low bits).
__device__ __forceinline__ uint32_t bytes_at_least(uint32_t c, uint32_t add4, bool hi) {
    const uint32_t s = (c & 0x7f7f7f7fu) + add4;
    return (hi ? (c & s) : (c | s)) & 0x80808080u;
}

struct ExtractArgs {
    const uint32_t *dense;  // mb rows of row_words words
    int64_t mb, n, row_words, q0;
    int32_t thr;            // keep ids whose count is >= thr
    const int64_t *off;     // optional: output of query q at [off[q], off[q+1]) ...
    int64_t cap;            // ... else at [q cap, (q+1) cap)
    int32_t *out_ids;
    uint8_t *out_counts;    // optional
    int32_t *out_n;         // per query: ids kept (all of them, even past the capacity)
    // optional: work items of the candidate search (k_cand_knn)
    int2 *items;
    uint32_t *n_items;
    int32_t chunk;
    int32_t *done;
};

// One block per row: the ids whose count passes the threshold, ascending,
// with their counts.  The row is read 4,096 counters at a time; a block-wide
// prefix sum over the threads' hit counts places every hit.
__global__ void __launch_bounds__(SH_THREADS) k_extract(const ExtractArgs a) {
    __shared__ int s_warp[SH_WARPS];
    __shared__ int64_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool hi = a.thr > 128;
    const uint32_t add4 = uint32_t(hi ? 256 - a.thr : 128 - a.thr) * 0x01010101u;
    const int64_t n16 = a.row_words >> 2;
    for (int64_t r = blockIdx.x; r < a.mb; r += gridDim.x) {
        const int64_t q = a.q0 + r;
        const uint4 *row = reinterpret_cast<const uint4 *>(a.dense + r * a.row_words);
        const int64_t obase = a.off != nullptr ? a.off[q] : q * a.cap;
        const int64_t ocap = a.off != nullptr ? a.off[q + 1] - a.off[q] : a.cap;
        if (threadIdx.x == 0) s_base = 0;
        __syncthreads();
        for (int64_t t0 = 0; t0 < n16; t0 += SH_THREADS) {
            const int64_t w = t0 + threadIdx.x;
            const uint4 c = w < n16 ? row[w] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
            uint32_t h[4];
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                h[u] = bytes_at_least(cw[u], add4, hi);
                cnt += __popc(h[u]);
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_warp[warp] = incl;
            __syncthreads();
            int before = 0, total = 0;
            for (int i = 0; i < SH_WARPS; ++i) {
                before += i < warp ? s_warp[i] : 0;
                total += s_warp[i];
            }
            int64_t pos = s_base + before + incl - cnt;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                uint32_t b = h[u];
                while (b != 0u) {
                    const int byte = (__ffs(int(b)) - 1) >> 3;
                    b &= b - 1u;
                    const int64_t id = 16 * w + 4 * u + byte;
                    if (id < a.n && pos < ocap) {
                        a.out_ids[obase + pos] = int32_t(id);
                        if (a.out_counts != nullptr) a.out_counts[obase + pos] = uint8_t(cw[u] >> (8 * byte));
                    }
                    ++pos;
                }
            }
            __syncthreads();  // every thread has read s_base and s_warp
            if (threadIdx.x == 0) s_base += total;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int c = int(s_base);
            a.out_n[q] = c;
            if (a.items != nullptr) {
                const int cc = int(std::min<int64_t>(c, ocap));
                const int nch = item_count(cc, item_size(cc, a.chunk));
                const uint32_t b0 = atomicAdd(a.n_items, uint32_t(nch));
                for (int j = 0; j < nch; ++j) a.items[b0 + j] = make_int2(int32_t(q), j);
                a.done[q] = 0;
            }
        }
        __syncthreads();
    }
}

int grid_for(int64_t work) { return int(std::max<int64_t>(1, std::min<int64_t>(work, 152 * 8))); }

}  // namespace
}  // namespace mrpt

using namespace mrpt;

namespace {

bool all_device(std::initializer_list<const void *> ptrs) {
    for (const void *p : ptrs)
        if (p != nullptr && !is_device_ptr(p)) return false;
    return true;
}

// Queries per batch of dense vote rows.
int64_t dense_batch(const mrpt_index *idx, int64_t m, int64_t row_words) {
    const int64_t per = row_words * 4;
    return std::max<int64_t>(1, std::min<int64_t>(m, int64_t(kDenseBudget) / per));
}

}  // namespace

extern "C" int mrpt_vote_counts(mrpt_index *idx, const float *Q, int64_t m, int32_t n_trees, int64_t cap,
                                int32_t *out_nnz, int32_t *out_ids, uint8_t *out_counts) {
    clear_error();
    if (!idx) {
        set_error("mrpt_vote_counts: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t T_use = n_trees > 0 ? n_trees : idx->T;
    const int64_t leaf_max = (idx->n + idx->L - 1) / idx->L;
    const int64_t bound = std::min<int64_t>(int64_t(T_use) * leaf_max, idx->n);
    if (m < 0 || T_use > idx->T || (m > 0 && (!Q || !out_nnz || !out_ids || !out_counts))) {
        set_error("mrpt_vote_counts: invalid argument (need m >= 0, n_trees <= T, non-NULL buffers)");
        return MRPT_ERR_INVALID_ARG;
    }
    if (cap < bound) {
        set_error("mrpt_vote_counts: cap must be at least min(n_trees ceil(n / 2^l), n) = " +
                  std::to_string(bound));
        return MRPT_ERR_INVALID_ARG;
    }
    if (m == 0) return MRPT_OK;
    if (!all_device({Q, out_nnz, out_ids, out_counts})) {
        set_error("mrpt_vote_counts: Q and the outputs must be device memory");
        return MRPT_ERR_INVALID_ARG;
    }
    cudaStream_t s = idx->stream;
    const int64_t row_words = ((idx->n + 15) / 16) * 4;
    const int64_t mb = dense_batch(idx, m, row_words);
    const size_t leaf_b = (size_t(mb) * size_t(T_use) * 4 + 255) & ~size_t(255);
    int rc = idx->shard.ensure(leaf_b + size_t(mb) * size_t(row_words) * 4, "vote count rows");
    if (rc) return rc;
    int32_t *leaf = static_cast<int32_t *>(idx->shard.ptr);
    uint32_t *dense = reinterpret_cast<uint32_t *>(static_cast<char *>(idx->shard.ptr) + leaf_b);
    for (int64_t q0 = 0; q0 < m; q0 += mb) {
        const int64_t mq = std::min(mb, m - q0);
        QueryLaunch ql{};
        ql.Q = Q + q0 * idx->d;
        ql.m = mq;
        ql.n_trees = T_use;
        ql.leaf = leaf;
        if ((rc = launch_route_only(idx, ql))) return rc;
        MRPT_CUDA_TRY(cudaMemsetAsync(dense, 0, size_t(mq) * size_t(row_words) * 4, s));
        k_dense_votes<<<grid_for(mq * T_use), SH_THREADS, 0, s>>>(leaf, T_use, idx->leaf_off, idx->leaf_ids,
                                                                  idx->n, mq, row_words, dense);
        MRPT_CUDA_TRY(cudaGetLastError());
        ExtractArgs a{};
        a.dense = dense;
        a.mb = mq;
        a.n = idx->n;
        a.row_words = row_words;
        a.q0 = q0;
        a.thr = 1;
        a.cap = cap;
        a.out_ids = out_ids;
        a.out_counts = out_counts;
        a.out_n = out_nnz;
        k_extract<<<grid_for(mq), SH_THREADS, 0, s>>>(a);
        MRPT_CUDA_TRY(cudaGetLastError());
    }
    return MRPT_OK;
}

extern "C" int mrpt_query_from_counts(mrpt_index *idx, const float *Q, int64_t m, int32_t k, int32_t v,
                                      const int64_t *off, const int32_t *ids, const uint8_t *counts,
                                      const mrpt_query_opts *opts, int32_t *out_ids, float *out_dists) {
    clear_error();
    if (!idx) {
        set_error("mrpt_query_from_counts: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t precision = opts ? opts->precision : MRPT_PREC_FP32;
    const int32_t margin = (opts && precision != MRPT_PREC_FP32) ? opts->margin : 0;
    if (m < 0 || (m > 0 && (!Q || !off || !out_ids || !out_dists)) || k < 1 || k > MRPT_MAX_K || v < 1 ||
        v > MRPT_MAX_TREES || (opts && (opts->chunk < 0 || opts->ring < 0)) ||
        (precision != MRPT_PREC_FP32 && precision != MRPT_PREC_BF16 && precision != MRPT_PREC_FP8) ||
        (precision == MRPT_PREC_BF16 && !idx->Xb) || (precision == MRPT_PREC_FP8 && !idx->X8) || margin < 0 ||
        k + margin > MRPT_MAX_K) {
        set_error("mrpt_query_from_counts: invalid argument (need m >= 0, non-NULL buffers, 1 <= k <= " +
                  std::to_string(MRPT_MAX_K) + ", 1 <= v <= " + std::to_string(MRPT_MAX_TREES) +
                  ", a precision whose copy exists, 0 <= margin, k + margin <= " + std::to_string(MRPT_MAX_K) +
                  ")");
        return MRPT_ERR_INVALID_ARG;
    }
    if (m == 0) return MRPT_OK;
    if (!all_device({Q, off, ids, counts, out_ids, out_dists})) {
        set_error("mrpt_query_from_counts: every buffer must be device memory");
        return MRPT_ERR_INVALID_ARG;
    }
    cudaStream_t s = idx->stream;
    // the list lengths bound |S| per query and size the work items
    std::vector<int64_t> h_off(size_t(m) + 1);
    MRPT_CUDA_TRY(cudaMemcpyAsync(h_off.data(), off, h_off.size() * 8, cudaMemcpyDeviceToHost, s));
    MRPT_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t longest = 0;
    for (int64_t q = 0; q < m; ++q) {
        const int64_t len = h_off[size_t(q) + 1] - h_off[size_t(q)];
        if (len < 0 || h_off[size_t(q)] < 0) {
            set_error("mrpt_query_from_counts: off must be non-decreasing from 0");
            return MRPT_ERR_INVALID_ARG;
        }
        longest = std::max(longest, len);
    }
    if (m > 0 && (ids == nullptr || counts == nullptr) && h_off[size_t(m)] > 0) {
        set_error("mrpt_query_from_counts: ids and counts are NULL but the lists are not empty");
        return MRPT_ERR_INVALID_ARG;
    }
    const int64_t total = h_off[size_t(m)];
    const int64_t ks = int64_t(k) + margin;
    int32_t chunk = int32_t(std::max<int64_t>(precision != MRPT_PREC_FP32 ? 32 : 64, ((2 * ks + 31) / 32) * 32));
    if (opts && opts->chunk > 0) chunk = int32_t(std::max<int64_t>(opts->chunk, ks));
    const int32_t max_items_q =
        int32_t(std::max<int64_t>(1, std::min<int64_t>((longest + chunk - 1) / chunk, CAND_ITEMS_MAX)));
    const int64_t row_words = ((idx->n + 15) / 16) * 4;
    const int64_t mb = dense_batch(idx, m, row_words);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t ctr_b = 256, cand_b = up(size_t(std::max<int64_t>(total, 1)) * 4), n_b = up(size_t(m) * 4),
                 it_b = up(size_t(m) * size_t(max_items_q) * 8),
                 part_b = up(size_t(m) * size_t(max_items_q) * size_t(ks) * 4),
                 dense_b = up(size_t(mb) * size_t(row_words) * 4);
    int rc = idx->shard.ensure(ctr_b + cand_b + 2 * n_b + it_b + 2 * part_b + dense_b, "counts query scratch");
    if (rc) return rc;
    char *base = static_cast<char *>(idx->shard.ptr);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(base);
    int32_t *cand = reinterpret_cast<int32_t *>(base + ctr_b);
    int32_t *ncand = reinterpret_cast<int32_t *>(base + ctr_b + cand_b);
    int32_t *done = reinterpret_cast<int32_t *>(base + ctr_b + cand_b + n_b);
    int2 *items = reinterpret_cast<int2 *>(base + ctr_b + cand_b + 2 * n_b);
    float *part_d = reinterpret_cast<float *>(base + ctr_b + cand_b + 2 * n_b + it_b);
    int32_t *part_i = reinterpret_cast<int32_t *>(base + ctr_b + cand_b + 2 * n_b + it_b + part_b);
    uint32_t *dense = reinterpret_cast<uint32_t *>(base + ctr_b + cand_b + 2 * n_b + it_b + 2 * part_b);
    MRPT_CUDA_TRY(cudaMemsetAsync(ctr, 0, ctr_b, s));
    for (int64_t q0 = 0; q0 < m; q0 += mb) {
        const int64_t mq = std::min(mb, m - q0);
        MRPT_CUDA_TRY(cudaMemsetAsync(dense, 0, size_t(mq) * size_t(row_words) * 4, s));
        if (total > 0) {
            k_sparse_to_dense<<<grid_for(mq), SH_THREADS, 0, s>>>(off, ids, counts, q0, mq, idx->n, row_words,
                                                                  dense);
            MRPT_CUDA_TRY(cudaGetLastError());
        }
        ExtractArgs a{};
        a.dense = dense;
        a.mb = mq;
        a.n = idx->n;
        a.row_words = row_words;
        a.q0 = q0;
        a.thr = v;
        a.off = off;
        a.out_ids = cand;
        a.out_n = ncand;
        a.items = items;
        a.n_items = ctr + 5;
        a.chunk = chunk;
        a.done = done;
        k_extract<<<grid_for(mq), SH_THREADS, 0, s>>>(a);
        MRPT_CUDA_TRY(cudaGetLastError());
    }
    // the exact search on S (Algorithm 4's knn), as in mrpt_query
    QueryLaunch ql{};
    ql.Q = Q;
    ql.m = m;
    ql.k = k;
    ql.v = v;
    ql.out_ids = out_ids;
    ql.out_dists = out_dists;
    ql.cand_list = cand;
    ql.cand_off = off;
    ql.capq = INT32_MAX;
    ql.ncand = ncand;
    ql.items = items;
    ql.chunk = chunk;
    ql.max_items_q = max_items_q;
    ql.done = done;
    ql.part_d = part_d;
    ql.part_i = part_i;
    ql.precision = precision;
    ql.margin = margin;
    ql.ring = (opts && opts->ring > 0) ? std::min<int32_t>(std::max<int32_t>(opts->ring, 2), 16) : 0;
    ql.counters = ctr;
    return launch_search_only(idx, ql);
}
