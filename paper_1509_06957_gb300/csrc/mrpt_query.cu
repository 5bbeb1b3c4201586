// Query phase (Sec. III, Algorithms 3-4) on sm_103a.
//
//   k_query_route   p = q^T R for every tree and level (Algorithm 3), then
//                   the descent p[level] <= split -> left.  A block stages up
//                   to 32 queries in shared memory; one thread per (query,
//                   tree), lanes of a warp share trees.
//   k_vote_search   persistent blocks take queries from an atomic counter.
//                   Per query: 8-bit vote counters for a chunk of point ids
//                   in shared memory, incremented by warp-wide passes over
//                   each tree's leaf (Algorithm 4's vote loop); points with
//                   at least v votes are compacted into a candidate buffer
//                   (S of Sec. III-A); a warp per candidate computes the
//                   float32 squared distance with 128-bit loads and keeps a
//                   per-warp sorted top-k in registers; the warps' lists are
//                   merged by rank (knn(q, k, S) of Algorithm 4).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "mrpt_internal.cuh"

namespace mrpt {

// ------------------------------------------------------------- routing ----

// One thread per (query, tree): lane = query (QB = 32 queries per tile, or
// QB < 32 queries x 32/QB trees per warp when d is large).  Work items are
// (query tile, group of ROUTE_TREES_PER_ITEM trees); a persistent block
// takes a contiguous range of items, so it stages a query tile once and
// walks its tree groups.  All lanes that share a tree read the same
// nonzero (dim, val) -- a broadcast load -- and take their query's
// component from shared memory (odd row stride: no bank conflicts).  Each
// projection is an fmaf chain in ascending dimension from +0.0f, followed by
// the descent p <= split -> left (Algorithm 3).
constexpr int ROUTE_TREES_PER_ITEM = 16;

template <int QB>
__global__ void __launch_bounds__(512) k_query_route(
    const float *__restrict__ Q, int64_t m, int32_t d, int32_t T_use, int32_t l, int64_t L,
    const int32_t *__restrict__ col_off, const int32_t *__restrict__ dim,
    const float *__restrict__ val, const float *__restrict__ split, int32_t *__restrict__ leaf,
    float *__restrict__ proj, uint32_t *__restrict__ status, int64_t n_items) {
    extern __shared__ float qs[];  // QB x (d | 1)
    const int stride = d | 1;
    constexpr int G = 32 / QB;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int qq = lane % QB;
    const int g = lane / QB;
    const float *qrow = qs + qq * stride;
    const int64_t inner = L - 1;
    const int ncols = T_use * l;
    const int groups = (T_use + ROUTE_TREES_PER_ITEM - 1) / ROUTE_TREES_PER_ITEM;
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0;
    // contiguous item range of this block
    const int64_t per = n_items / gridDim.x, extra = n_items % gridDim.x;
    const int64_t bx = blockIdx.x;
    const int64_t it0 = bx * per + (bx < extra ? bx : extra);
    const int64_t it1 = it0 + per + (int64_t(blockIdx.x) < extra ? 1 : 0);
    int64_t staged = -1;
    for (int64_t it = it0; it < it1; ++it) {
        const int64_t tile = it / groups;
        const int grp = int(it - tile * groups);
        const int64_t q0 = tile * QB;
        const int nq = int((m - q0) < QB ? (m - q0) : int64_t(QB));
        if (tile != staged) {
            __syncthreads();  // the previous tile is no longer read
            bool bad = false;
            for (int r = warp; r < QB; r += nwarps) {
                float *dst = qs + r * stride;
                if (r < nq) {
                    const float *src = Q + (q0 + r) * d;
                    if (vec) {
                        for (int c4 = lane; c4 < (d >> 2); c4 += 32) {
                            const float4 x = __ldg(reinterpret_cast<const float4 *>(src) + c4);
                            bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
                            dst[4 * c4 + 0] = x.x;
                            dst[4 * c4 + 1] = x.y;
                            dst[4 * c4 + 2] = x.z;
                            dst[4 * c4 + 3] = x.w;
                        }
                    } else {
                        for (int c = lane; c < d; c += 32) {
                            const float x = __ldg(src + c);
                            bad |= !isfinite(x);
                            dst[c] = x;
                        }
                    }
                } else {
                    for (int c = lane; c < d; c += 32) dst[c] = 0.f;
                }
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, STATUS_NONFINITE_QUERY);
            __syncthreads();
            staged = tile;
        }
        const bool live = qq < nq;
        const int t_begin = grp * ROUTE_TREES_PER_ITEM;
        const int t_end = min(T_use, t_begin + ROUTE_TREES_PER_ITEM);
        for (int tb = t_begin + warp * G; tb < t_end; tb += nwarps * G) {
            const int t = tb + g;
            const bool tree_ok = t < t_end;
            const int tt = tree_ok ? t : t_begin;
            const float *sp = split + int64_t(tt) * inner;
            int64_t node = 0;
            for (int j = 0; j < l; ++j) {
                const int c = tt * l + j;
                const int e1 = __ldg(col_off + c + 1);
                int e = __ldg(col_off + c);
                float acc = 0.0f;
                for (; e + 4 <= e1; e += 4) {
                    const int d0 = __ldg(dim + e), d1 = __ldg(dim + e + 1);
                    const int d2 = __ldg(dim + e + 2), d3 = __ldg(dim + e + 3);
                    const float v0 = __ldg(val + e), v1 = __ldg(val + e + 1);
                    const float v2 = __ldg(val + e + 2), v3 = __ldg(val + e + 3);
                    const float x0 = qrow[d0], x1 = qrow[d1], x2 = qrow[d2], x3 = qrow[d3];
                    acc = __fmaf_rn(x0, v0, acc);
                    acc = __fmaf_rn(x1, v1, acc);
                    acc = __fmaf_rn(x2, v2, acc);
                    acc = __fmaf_rn(x3, v3, acc);
                }
                for (; e < e1; ++e) acc = __fmaf_rn(qrow[__ldg(dim + e)], __ldg(val + e), acc);
                if (proj != nullptr && live && tree_ok) proj[(q0 + qq) * ncols + c] = acc;
                node = 2 * node + 1 + (acc > __ldg(sp + node) ? 1 : 0);
            }
            if (live && tree_ok) leaf[(q0 + qq) * T_use + t] = int32_t(node - inner);
        }
    }
}

// ---------------------------------------------------------- vote search ----

constexpr int VS_THREADS = 256;
constexpr int VS_WARPS = VS_THREADS / 32;
constexpr int CH_WORDS = 16384;          // 64 KB: 8-bit counters for 65,536 ids
constexpr int64_t CH_IDS = int64_t(CH_WORDS) * 4;
constexpr int32_t SENTINEL_ID = 0x7fffffff;

__device__ __forceinline__ bool pair_less(float da, int32_t ia, float db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

// A warp's k smallest (distance, id) pairs, sorted ascending; entry
// r*32 + lane lives in lane `lane`, slot r.
template <int KR>
struct WarpTopK {
    float d[KR];
    int32_t i[KR];
    float thr_d;
    int32_t thr_i;

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            d[r] = INFINITY;
            i[r] = SENTINEL_ID;
        }
        thr_d = INFINITY;
        thr_i = SENTINEL_ID;
    }

    // nd/ni are warp-uniform.
    __device__ __forceinline__ void insert(float nd, int32_t ni, int k, int lane) {
        if (!pair_less(nd, ni, thr_d, thr_i)) return;
        int pos = 0;
#pragma unroll
        for (int r = 0; r < KR; ++r)
            pos += __popc(__ballot_sync(0xffffffffu, pair_less(d[r], i[r], nd, ni)));
#pragma unroll
        for (int r = KR - 1; r >= 0; --r) {
            float ud = __shfl_up_sync(0xffffffffu, d[r], 1);
            int32_t ui = __shfl_up_sync(0xffffffffu, i[r], 1);
            float pd = INFINITY;
            int32_t pi = SENTINEL_ID;
            if (r > 0) {
                pd = __shfl_sync(0xffffffffu, d[r > 0 ? r - 1 : 0], 31);
                pi = __shfl_sync(0xffffffffu, i[r > 0 ? r - 1 : 0], 31);
            }
            if (lane == 0) {
                ud = pd;
                ui = pi;
            }
            const int e = r * 32 + lane;
            if (e > pos) {
                d[r] = ud;
                i[r] = ui;
            } else if (e == pos) {
                d[r] = nd;
                i[r] = ni;
            }
        }
        const int rr = (k - 1) >> 5;
        float td = d[0];
        int32_t ti = i[0];
#pragma unroll
        for (int r = 1; r < KR; ++r)
            if (r == rr) {
                td = d[r];
                ti = i[r];
            }
        thr_d = __shfl_sync(0xffffffffu, td, (k - 1) & 31);
        thr_i = __shfl_sync(0xffffffffu, ti, (k - 1) & 31);
    }
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Squared Euclidean distances between the staged query and R rows (R <= 2):
// every lane keeps up to 4 float4 loads per row in flight before it
// accumulates, then the warp reduces each row's partial sums.
template <int R>
__device__ __forceinline__ void rows_sq_dist(const float4 *const (&rows)[2],
                                             const float4 *__restrict__ q4, int nv4, int lane,
                                             float (&out)[2]) {
    float acc[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r][0] = acc[r][1] = 0.f;
    for (int base = lane; base < nv4; base += 128) {
        float4 x[R][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = base + 32 * u;
#pragma unroll
            for (int r = 0; r < R; ++r)
                x[r][u] = (j < nv4) ? __ldg(rows[r] + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = base + 32 * u;
            if (j < nv4) {
                const float4 q = q4[j];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float dx = q.x - x[r][u].x, dy = q.y - x[r][u].y;
                    const float dz = q.z - x[r][u].z, dw = q.w - x[r][u].w;
                    acc[r][0] = __fmaf_rn(dx, dx, acc[r][0]);
                    acc[r][1] = __fmaf_rn(dy, dy, acc[r][1]);
                    acc[r][0] = __fmaf_rn(dz, dz, acc[r][0]);
                    acc[r][1] = __fmaf_rn(dw, dw, acc[r][1]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = warp_sum(acc[r][0] + acc[r][1]);
}

struct VoteSearchArgs {
    const float *X;
    int64_t n;
    int32_t dpad;
    const float *Q;
    int64_t m;
    int32_t d;
    const int32_t *leaf_of_q;
    int32_t T_use;
    const int32_t *leaf_off;
    const int32_t *leaf_ids;
    int32_t k, v;
    int32_t *out_ids;
    float *out_dists;
    uint8_t *dbg_votes;
    int64_t *dbg_ncand;
    int32_t *dbg_cand;
    int64_t cand_cap;
    uint32_t *work;
    int32_t cnt_words;     // counter words per chunk (<= CH_WORDS, multiple of 4)
    int32_t region_bytes;  // bytes of the counter / merge region (multiple of 16)
    const int32_t *qlist;        // optional: process only these queries ...
    const uint32_t *qlist_len;   // ... this many of them (read on the device)
};

// Per warp: a buffer of emitted candidates waiting for their distances.
constexpr int WBUF = 256;

// One block per query at a time (queries taken from an atomic counter).
//   1. clear the 8-bit vote counters of the id chunk [c0, c0 + CH_IDS);
//   2. every warp walks the leaves of its trees (t = warp, warp + W, ...),
//      128 ids per step, and adds one vote per id with a shared-memory
//      atomic; the lane whose increment takes a count from v-1 to v emits
//      the id (Algorithm 4: "if votes[point] = v then S <- S u {point}");
//   3. a warp computes the exact distances of the ids it emitted itself
//      (64 or more at a time) and keeps them in its own top-k -- warps
//      never wait for each other between the clear and the merge;
//   4. the warps' top-k lists are merged by rank.
// Emission is final (votes only grow), so a candidate's distance can be
// computed as soon as it is emitted.  Ids above the chunk are left for the
// next chunk through per-tree cursors (leaves list ids in ascending order).
template <int KR>
__global__ void __launch_bounds__(VS_THREADS, 3) k_vote_search(const VoteSearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);                        // a.cnt_words
    float *qv = reinterpret_cast<float *>(smem + size_t(a.region_bytes));      // dpad
    int32_t *wbuf = reinterpret_cast<int32_t *>(qv + a.dpad);                  // VS_WARPS * WBUF
    int32_t *cur = wbuf + VS_WARPS * WBUF;                                      // T_use
    int32_t *lend = cur + a.T_use;                                              // T_use
    int32_t *cend = lend + a.T_use;                                             // T_use
    // merge area (aliases the counters once voting is over)
    float *md = reinterpret_cast<float *>(smem);                                // VS_WARPS * KR*32
    int32_t *mi = reinterpret_cast<int32_t *>(smem + VS_WARPS * KR * 32 * 4);
    __shared__ int64_t s_q;
    __shared__ unsigned long long s_total;
    __shared__ int s_real[VS_WARPS];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nv4 = a.dpad >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(qv);
    const float4 *X4 = reinterpret_cast<const float4 *>(a.X);
    const int k = a.k;
    const uint32_t vm1 = uint32_t(a.v - 1);
    const bool track = (a.dbg_ncand != nullptr) || (a.dbg_cand != nullptr);
    constexpr int K2 = KR * 32;
    int32_t *mybuf = wbuf + warp * WBUF;

    for (;;) {
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            int64_t q = -1;
            if (a.qlist != nullptr) {
                if (w < *a.qlist_len) q = a.qlist[w];
            } else if (int64_t(w) < a.m) {
                q = int64_t(w);
            }
            s_q = q;
            s_total = 0ull;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;

        for (int i = tid; i < a.dpad; i += VS_THREADS) qv[i] = (i < a.d) ? a.Q[qi * a.d + i] : 0.f;
        for (int t = tid; t < a.T_use; t += VS_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * a.T_use + t];
            cur[t] = a.leaf_off[lf];
            lend[t] = a.leaf_off[lf + 1];
        }
        WarpTopK<KR> top;
        top.init();

        // exact distances of this warp's buffered candidates
        auto drain = [&](int nb) {
            __syncwarp();
            int j = 0;
            for (; j + 1 < nb; j += 2) {
                const int32_t id0 = mybuf[j];
                const int32_t id1 = mybuf[j + 1];
                const float4 *rows[2] = {X4 + int64_t(id0) * nv4, X4 + int64_t(id1) * nv4};
                float dd[2];
                rows_sq_dist<2>(rows, q4, nv4, lane, dd);
                top.insert(dd[0], id0, k, lane);
                top.insert(dd[1], id1, k, lane);
            }
            if (j < nb) {
                const int32_t id0 = mybuf[j];
                const float4 *rows[2] = {X4 + int64_t(id0) * nv4, X4 + int64_t(id0) * nv4};
                float dd[2];
                rows_sq_dist<1>(rows, q4, nv4, lane, dd);
                top.insert(dd[0], id0, k, lane);
            }
            __syncwarp();
        };

        for (int64_t c0 = 0; c0 < a.n; c0 += CH_IDS) {
            const int64_t wleft = (a.n - c0 + 3) >> 2;
            const int nwords = int(wleft < a.cnt_words ? wleft : int64_t(a.cnt_words));
            {
                uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
                const int n4 = (nwords + 3) >> 2;
                for (int w = tid; w < n4; w += VS_THREADS) c4[w] = make_uint4(0u, 0u, 0u, 0u);
            }
            const int64_t lim = c0 + CH_IDS;
            // end of each tree's ids inside this chunk: leaves list ids in
            // ascending order, so it is a lower bound of `lim`
            for (int t = tid; t < a.T_use; t += VS_THREADS) {
                int32_t lo = cur[t], hi = lend[t];
                if (lim < a.n) {
                    const int32_t *ids = a.leaf_ids + int64_t(t) * a.n;
                    while (lo < hi) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (int64_t(__ldg(ids + mid)) < lim)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    cend[t] = lo;
                } else {
                    cend[t] = hi;
                }
            }
            __syncthreads();
            int nb = 0;
            // the warp's tiles (128 consecutive ids of one tree's leaf) in
            // order; the next tile is loaded while the current one votes
            int t = warp;
            int32_t p = 0, e = 0;
            while (t < a.T_use) {
                p = cur[t];
                e = cend[t];
                if (p < e) break;
                t += VS_WARPS;
            }
            int32_t id[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t i = p + 32 * u + lane;
                id[u] = (t < a.T_use && i < e) ? __ldg(a.leaf_ids + int64_t(t) * a.n + i) : -1;
            }
            while (t < a.T_use) {
                // position and prefetch of the next tile
                int tn = t;
                int32_t pn = p + 128, en = e;
                if (pn >= en) {
                    if (lane == 0) cur[t] = en;
                    tn = t + VS_WARPS;
                    while (tn < a.T_use) {
                        pn = cur[tn];
                        en = cend[tn];
                        if (pn < en) break;
                        tn += VS_WARPS;
                    }
                }
                int32_t idn[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t i = pn + 32 * u + lane;
                    idn[u] = (tn < a.T_use && i < en) ? __ldg(a.leaf_ids + int64_t(tn) * a.n + i) : -1;
                }
                // votes of the current tile
                // every atomic of the tile is issued before any result is used
                uint32_t olds[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    olds[u] = 0u;
                    if (id[u] >= 0) {
                        const uint32_t off = uint32_t(int64_t(id[u]) - c0);
                        const uint32_t sh = (off & 3u) * 8u;
                        olds[u] = atomicAdd(&cnt[off >> 2], 1u << sh) >> sh;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool emit = id[u] >= 0 && (olds[u] & 0xffu) == vm1;
                    const unsigned em = __ballot_sync(0xffffffffu, emit);
                    if (em) {
                        if (emit) mybuf[nb + __popc(em & lt)] = id[u];
                        if (track) {
                            unsigned long long base = 0;
                            if (lane == 0) base = atomicAdd(&s_total, (unsigned long long)__popc(em));
                            base = __shfl_sync(0xffffffffu, base, 0);
                            if (emit && a.dbg_cand != nullptr) {
                                const int64_t slot = int64_t(base) + __popc(em & lt);
                                if (slot < a.cand_cap) a.dbg_cand[qi * a.cand_cap + slot] = id[u];
                            }
                        }
                        nb += __popc(em);
                    }
                }
                if (nb >= 64) {
                    drain(nb);
                    nb = 0;
                }
                t = tn;
                p = pn;
                e = en;
#pragma unroll
                for (int u = 0; u < 4; ++u) id[u] = idn[u];
            }
            if (nb > 0) drain(nb);
            __syncthreads();
            if (a.dbg_votes != nullptr) {
                for (int w = tid; w < nwords; w += VS_THREADS) {
                    const uint32_t word = cnt[w];
                    for (int b = 0; b < 4; ++b) {
                        const int64_t id = c0 + 4 * int64_t(w) + b;
                        if (id < a.n) a.dbg_votes[qi * a.n + id] = uint8_t((word >> (8 * b)) & 0xffu);
                    }
                }
                __syncthreads();
            }
        }
        // ---- merge the warps' lists by rank
        {
            int real = 0;
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int e = r * 32 + lane;
                md[warp * K2 + e] = top.d[r];
                mi[warp * K2 + e] = top.i[r];
                real += (e < k && top.i[r] != SENTINEL_ID) ? 1 : 0;
            }
            real = __reduce_add_sync(0xffffffffu, real);
            if (lane == 0) s_real[warp] = real;
        }
        __syncthreads();
        int all_real = 0;
        for (int w = 0; w < VS_WARPS; ++w) all_real += s_real[w];
        const int filled = min(all_real, k);
        int32_t *oi = a.out_ids + qi * k;
        float *od = a.out_dists + qi * k;
        for (int e = filled + tid; e < k; e += VS_THREADS) {
            oi[e] = -1;
            od[e] = INFINITY;
        }
        for (int x = tid; x < VS_WARPS * k; x += VS_THREADS) {
            const int w = x / k;
            const int e = x - w * k;
            const int32_t id = mi[w * K2 + e];
            if (id == SENTINEL_ID) continue;
            const float dd = md[w * K2 + e];
            int rank = e;
            for (int w2 = 0; w2 < VS_WARPS && rank < k; ++w2) {
                if (w2 == w) continue;
                // entries of list w2 (first k) strictly below (dd, id)
                int lo = 0, hi = k;
                const float *ld = md + w2 * K2;
                const int32_t *li = mi + w2 * K2;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (pair_less(ld[mid], li[mid], dd, id))
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                rank += lo;
            }
            if (rank < k) {
                oi[rank] = id;
                od[rank] = sqrtf(dd);
            }
        }
        if (a.dbg_ncand != nullptr && tid == 0) a.dbg_ncand[qi] = int64_t(s_total);
        __syncthreads();
    }
}

// ------------------------------------------------- vote / emit + search ----
//
// The batched path splits the query in two kernels:
//   k_vote_emit  votes (as in k_vote_search) and writes each query's
//                candidate set S to a per-query list in global memory; it
//                carries no distance state, so a block has 16 warps.
//   k_cand_knn   one warp per query: exact distances of the listed
//                candidates (128-bit row loads, two rows in flight) and the
//                warp's sorted top-k, written straight to the output row.
// Queries whose |S| exceeds the list capacity are appended to an overflow
// list and answered by k_vote_search, which needs no list.

constexpr int VE_THREADS = 512;
constexpr int VE_WARPS = VE_THREADS / 32;

struct VoteEmitArgs {
    int64_t n;
    const int32_t *leaf_of_q;
    int32_t T_use;
    const int32_t *leaf_off;
    const int32_t *leaf_ids;
    int64_t m;
    int32_t v;
    int32_t *cand;         // m x capq candidate ids
    int32_t capq;
    int32_t *ncand;        // m: |S|
    int32_t *overflow;     // queries with |S| > capq
    uint32_t *n_overflow;
    uint32_t *work;
    int32_t cnt_words;
    uint8_t *dbg_votes;
    int64_t *dbg_ncand;
    int32_t *dbg_cand;
    int64_t cand_cap;
};

__global__ void __launch_bounds__(VE_THREADS, 3) k_vote_emit(const VoteEmitArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // cnt_words
    int32_t *cur = reinterpret_cast<int32_t *>(cnt + a.cnt_words);
    int32_t *lend = cur + a.T_use;
    int32_t *cend = lend + a.T_use;
    __shared__ int64_t s_q;
    __shared__ int s_cnt;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t vm1 = uint32_t(a.v - 1);

    for (;;) {
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;
        for (int t = tid; t < a.T_use; t += VE_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * a.T_use + t];
            cur[t] = a.leaf_off[lf];
            lend[t] = a.leaf_off[lf + 1];
        }
        int32_t *clist = a.cand + qi * int64_t(a.capq);
        for (int64_t c0 = 0; c0 < a.n; c0 += CH_IDS) {
            const int64_t wleft = (a.n - c0 + 3) >> 2;
            const int nwords = int(wleft < a.cnt_words ? wleft : int64_t(a.cnt_words));
            {
                uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
                const int n4 = (nwords + 3) >> 2;
                for (int w = tid; w < n4; w += VE_THREADS) c4[w] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncthreads();  // cur/lend written, counters cleared
            const int64_t lim = c0 + CH_IDS;
            for (int t = tid; t < a.T_use; t += VE_THREADS) {
                int32_t lo = cur[t], hi = lend[t];
                if (lim < a.n) {
                    const int32_t *ids = a.leaf_ids + int64_t(t) * a.n;
                    while (lo < hi) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (int64_t(__ldg(ids + mid)) < lim)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    cend[t] = lo;
                } else {
                    cend[t] = hi;
                }
            }
            __syncthreads();
            // the warp's 128-id tiles, the next one loaded while the current
            // one votes
            int t = warp;
            int32_t p = 0, e = 0;
            while (t < a.T_use) {
                p = cur[t];
                e = cend[t];
                if (p < e) break;
                t += VE_WARPS;
            }
            int32_t id[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t i = p + 32 * u + lane;
                id[u] = (t < a.T_use && i < e) ? __ldg(a.leaf_ids + int64_t(t) * a.n + i) : -1;
            }
            while (t < a.T_use) {
                int tn = t;
                int32_t pn = p + 128, en = e;
                if (pn >= en) {
                    if (lane == 0) cur[t] = en;
                    tn = t + VE_WARPS;
                    while (tn < a.T_use) {
                        pn = cur[tn];
                        en = cend[tn];
                        if (pn < en) break;
                        tn += VE_WARPS;
                    }
                }
                int32_t idn[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t i = pn + 32 * u + lane;
                    idn[u] = (tn < a.T_use && i < en) ? __ldg(a.leaf_ids + int64_t(tn) * a.n + i) : -1;
                }
                uint32_t olds[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    olds[u] = 0u;
                    if (id[u] >= 0) {
                        const uint32_t off = uint32_t(int64_t(id[u]) - c0);
                        const uint32_t sh = (off & 3u) * 8u;
                        olds[u] = atomicAdd(&cnt[off >> 2], 1u << sh) >> sh;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // Algorithm 4: a point joins S when its count becomes v
                    const bool emit = id[u] >= 0 && (olds[u] & 0xffu) == vm1;
                    const unsigned em = __ballot_sync(0xffffffffu, emit);
                    if (em) {
                        int base = 0;
                        if (lane == 0) base = atomicAdd(&s_cnt, __popc(em));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (emit) {
                            const int slot = base + __popc(em & lt);
                            if (slot < a.capq) clist[slot] = id[u];
                            if (a.dbg_cand != nullptr && slot < a.cand_cap)
                                a.dbg_cand[qi * a.cand_cap + slot] = id[u];
                        }
                    }
                }
                t = tn;
                p = pn;
                e = en;
#pragma unroll
                for (int u = 0; u < 4; ++u) id[u] = idn[u];
            }
            __syncthreads();
            if (a.dbg_votes != nullptr) {
                for (int w = tid; w < nwords; w += VE_THREADS) {
                    const uint32_t word = cnt[w];
                    for (int b = 0; b < 4; ++b) {
                        const int64_t id2 = c0 + 4 * int64_t(w) + b;
                        if (id2 < a.n) a.dbg_votes[qi * a.n + id2] = uint8_t((word >> (8 * b)) & 0xffu);
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            const int c = s_cnt;
            a.ncand[qi] = c;
            if (a.dbg_ncand != nullptr) a.dbg_ncand[qi] = c;
            if (c > a.capq) a.overflow[atomicAdd(a.n_overflow, 1u)] = int32_t(qi);
        }
    }
}

constexpr int CK_THREADS = 256;
constexpr int CK_WARPS = CK_THREADS / 32;

struct CandKnnArgs {
    const float *X;
    int32_t dpad;
    const float *Q;
    int64_t m;
    int32_t d;
    const int32_t *cand;
    int32_t capq;
    const int32_t *ncand;
    int32_t k;
    int32_t *out_ids;
    float *out_dists;
    uint32_t *work;
};

template <int KR>
__global__ void __launch_bounds__(CK_THREADS) k_cand_knn(const CandKnnArgs a) {
    extern __shared__ __align__(16) float qsm[];  // CK_WARPS x dpad
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *qv = qsm + warp * a.dpad;
    const float4 *q4 = reinterpret_cast<const float4 *>(qv);
    const float4 *X4 = reinterpret_cast<const float4 *>(a.X);
    const int nv4 = a.dpad >> 2;
    const int k = a.k;
    for (;;) {
        int64_t qi = 0;
        if (lane == 0) qi = int64_t(atomicAdd(a.work, 1u));
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= a.m) break;
        const int c = a.ncand[qi];
        if (c > a.capq) continue;  // answered by the overflow pass
        for (int i = lane; i < a.dpad; i += 32) qv[i] = (i < a.d) ? a.Q[qi * a.d + i] : 0.f;
        __syncwarp();
        WarpTopK<KR> top;
        top.init();
        const int32_t *clist = a.cand + qi * int64_t(a.capq);
        for (int base = 0; base < c; base += 32) {
            const int32_t mine = (base + lane < c) ? __ldg(clist + base + lane) : 0;
            const int cb = min(32, c - base);
            int j = 0;
            for (; j + 1 < cb; j += 2) {
                const int32_t id0 = __shfl_sync(0xffffffffu, mine, j);
                const int32_t id1 = __shfl_sync(0xffffffffu, mine, j + 1);
                const float4 *rows[2] = {X4 + int64_t(id0) * nv4, X4 + int64_t(id1) * nv4};
                float dd[2];
                rows_sq_dist<2>(rows, q4, nv4, lane, dd);
                top.insert(dd[0], id0, k, lane);
                top.insert(dd[1], id1, k, lane);
            }
            if (j < cb) {
                const int32_t id0 = __shfl_sync(0xffffffffu, mine, j);
                const float4 *rows[2] = {X4 + int64_t(id0) * nv4, X4 + int64_t(id0) * nv4};
                float dd[2];
                rows_sq_dist<1>(rows, q4, nv4, lane, dd);
                top.insert(dd[0], id0, k, lane);
            }
        }
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            const int e = r * 32 + lane;
            if (e < k) {
                const bool real = top.i[r] != SENTINEL_ID;
                a.out_ids[qi * k + e] = real ? top.i[r] : -1;
                a.out_dists[qi * k + e] = real ? sqrtf(top.d[r]) : INFINITY;
            }
        }
        __syncwarp();
    }
}

// -------------------------------------------------------------- launch ----

namespace {

template <int QB>
cudaError_t launch_route(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const size_t smem = size_t(QB) * size_t(idx->d | 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_query_route<QB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_query_route<QB>, 512, smem);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, idx->device);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (ql.m + QB - 1) / QB;
    const int64_t groups = (ql.n_trees + ROUTE_TREES_PER_ITEM - 1) / ROUTE_TREES_PER_ITEM;
    const int64_t items = tiles * groups;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(items, int64_t(sms) * std::max(per_sm, 1)));
    k_query_route<QB><<<unsigned(blocks), 512, smem, s>>>(ql.Q, ql.m, idx->d, ql.n_trees, idx->l,
                                                         idx->L, idx->col_off, idx->dim, idx->val,
                                                         idx->split, ql.leaf, ql.proj, idx->status,
                                                         items);
    return cudaGetLastError();
}

// Shared-memory plan and arguments of k_vote_search.
template <int KR>
cudaError_t plan_vote(const mrpt_index *idx, const QueryLaunch &ql, uint32_t *work,
                      VoteSearchArgs &a, size_t &smem, int64_t &blocks) {
    // counters for min(n, CH_IDS) ids, rounded to 16 bytes; the same region
    // later holds the warps' top-k lists for the merge
    const int64_t ids_chunk = idx->n < CH_IDS ? idx->n : CH_IDS;
    const int cnt_words = int(((ids_chunk + 3) / 4 + 3) & ~int64_t(3));
    const size_t merge_bytes = size_t(VS_WARPS) * KR * 32 * 8;
    size_t region = std::max(size_t(cnt_words) * 4, merge_bytes);
    region = (region + 15) & ~size_t(15);
    smem = region + size_t(idx->dpad) * 4 + size_t(VS_WARPS) * WBUF * 4 + size_t(3 * ql.n_trees) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_vote_search<KR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vote_search<KR>, VS_THREADS, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, idx->device);
    if (e != cudaSuccess) return e;
    blocks = std::max<int64_t>(1, std::min<int64_t>(ql.m, int64_t(sms) * std::max(per_sm, 1)));
    a = VoteSearchArgs{};
    a.X = idx->X;
    a.n = idx->n;
    a.dpad = idx->dpad;
    a.Q = ql.Q;
    a.m = ql.m;
    a.d = idx->d;
    a.leaf_of_q = ql.leaf;
    a.T_use = ql.n_trees;
    a.leaf_off = idx->leaf_off;
    a.leaf_ids = idx->leaf_ids;
    a.k = ql.k;
    a.v = ql.v;
    a.out_ids = ql.out_ids;
    a.out_dists = ql.out_dists;
    a.dbg_votes = ql.votes;
    a.dbg_ncand = ql.n_cand;
    a.dbg_cand = ql.cand;
    a.cand_cap = ql.cand_cap;
    a.work = work;
    a.cnt_words = cnt_words;
    a.region_bytes = int(region);
    return cudaSuccess;
}

template <int KR>
cudaError_t launch_vote(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    VoteSearchArgs a;
    size_t smem = 0;
    int64_t blocks = 0;
    cudaError_t e = plan_vote<KR>(idx, ql, idx->status + 1, a, smem, blocks);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(idx->status + 1, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_vote_search<KR><<<unsigned(blocks), VS_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// As launch_vote, with the work counter at `work` (cleared here).
template <int KR>
cudaError_t launch_vote_with_counter(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s,
                                     uint32_t *work) {
    VoteSearchArgs a;
    size_t smem = 0;
    int64_t blocks = 0;
    cudaError_t e = plan_vote<KR>(idx, ql, work, a, smem, blocks);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_vote_search<KR><<<unsigned(blocks), VS_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

namespace {

cudaError_t launch_route_any(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    // as many queries per block (up to 32, one per lane) as fit in ~110 KB
    const int64_t per_q = int64_t(idx->d) * 4;
    if (per_q * 32 <= 110 * 1024) return launch_route<32>(idx, ql, s);
    if (per_q * 16 <= 110 * 1024) return launch_route<16>(idx, ql, s);
    if (per_q * 8 <= 160 * 1024) return launch_route<8>(idx, ql, s);
    if (per_q * 4 <= 160 * 1024) return launch_route<4>(idx, ql, s);
    if (per_q * 2 <= 200 * 1024) return launch_route<2>(idx, ql, s);
    return launch_route<1>(idx, ql, s);
}

cudaError_t launch_vote_emit(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const int64_t ids_chunk = idx->n < CH_IDS ? idx->n : CH_IDS;
    const int cnt_words = int(((ids_chunk + 3) / 4 + 3) & ~int64_t(3));
    const size_t smem = size_t(cnt_words) * 4 + size_t(3 * ql.n_trees) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_vote_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vote_emit, VE_THREADS, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, idx->device);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ql.m, int64_t(sms) * std::max(per_sm, 1)));
    VoteEmitArgs a{};
    a.n = idx->n;
    a.leaf_of_q = ql.leaf;
    a.T_use = ql.n_trees;
    a.leaf_off = idx->leaf_off;
    a.leaf_ids = idx->leaf_ids;
    a.m = ql.m;
    a.v = ql.v;
    a.cand = ql.cand_list;
    a.capq = ql.capq;
    a.ncand = ql.ncand;
    a.overflow = ql.overflow;
    a.n_overflow = idx->status + 3;
    a.work = idx->status + 1;
    a.cnt_words = cnt_words;
    a.dbg_votes = ql.votes;
    a.dbg_ncand = ql.n_cand;
    a.dbg_cand = ql.cand;
    a.cand_cap = ql.cand_cap;
    k_vote_emit<<<unsigned(blocks), VE_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KR>
cudaError_t launch_cand_knn(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const size_t smem = size_t(CK_WARPS) * size_t(idx->dpad) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_cand_knn<KR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cand_knn<KR>, CK_THREADS, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, idx->device);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>((ql.m + CK_WARPS - 1) / CK_WARPS, int64_t(sms) * std::max(per_sm, 1)));
    CandKnnArgs a{};
    a.X = idx->X;
    a.dpad = idx->dpad;
    a.Q = ql.Q;
    a.m = ql.m;
    a.d = idx->d;
    a.cand = ql.cand_list;
    a.capq = ql.capq;
    a.ncand = ql.ncand;
    a.k = ql.k;
    a.out_ids = ql.out_ids;
    a.out_dists = ql.out_dists;
    a.work = idx->status + 2;
    k_cand_knn<KR><<<unsigned(blocks), CK_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// k_vote_search over the overflow list (its length is read on the device).
template <int KR>
cudaError_t launch_overflow(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    VoteSearchArgs a;
    size_t smem = 0;
    int64_t blocks = 0;
    QueryLaunch q2 = ql;
    q2.votes = nullptr;
    q2.n_cand = nullptr;
    q2.cand = nullptr;
    cudaError_t e = plan_vote<KR>(idx, q2, idx->status + 4, a, smem, blocks);
    if (e != cudaSuccess) return e;
    a.qlist = ql.overflow;
    a.qlist_len = idx->status + 3;
    k_vote_search<KR><<<unsigned(blocks), VS_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int launch_query(mrpt_index *idx, const QueryLaunch &ql) {
    cudaStream_t s = idx->stream;
    if (ql.m == 0) return MRPT_OK;
    cudaError_t e;
    if (ql.stage_ms) {
        for (int i = 0; i < 4; ++i)
            if (!idx->ev[i]) MRPT_CUDA_TRY(cudaEventCreate(&idx->ev[i]));
        MRPT_CUDA_TRY(cudaEventRecord(idx->ev[0], s));
    }
    e = launch_route_any(idx, ql, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_query_route");
    if (ql.stage_ms) MRPT_CUDA_TRY(cudaEventRecord(idx->ev[1], s));
    const int kr = (ql.k + 31) / 32;
    if (ql.path == 1 || ql.cand_list == nullptr) {
        // one fused kernel
        if (kr <= 1)
            e = launch_vote<1>(idx, ql, s);
        else if (kr <= 2)
            e = launch_vote<2>(idx, ql, s);
        else if (kr <= 4)
            e = launch_vote<4>(idx, ql, s);
        else
            e = launch_vote<8>(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_vote_search");
        if (ql.stage_ms) MRPT_CUDA_TRY(cudaEventRecord(idx->ev[2], s));
    } else {
        // work counters [1] vote/emit, [2] candidate search, [3] overflow
        // length, [4] overflow pass
        MRPT_CUDA_TRY(cudaMemsetAsync(idx->status + 1, 0, 4 * sizeof(uint32_t), s));
        e = launch_vote_emit(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_vote_emit");
        if (ql.stage_ms) MRPT_CUDA_TRY(cudaEventRecord(idx->ev[2], s));
        if (kr <= 1)
            e = launch_cand_knn<1>(idx, ql, s);
        else if (kr <= 2)
            e = launch_cand_knn<2>(idx, ql, s);
        else if (kr <= 4)
            e = launch_cand_knn<4>(idx, ql, s);
        else
            e = launch_cand_knn<8>(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_cand_knn");
        if (kr <= 1)
            e = launch_overflow<1>(idx, ql, s);
        else if (kr <= 2)
            e = launch_overflow<2>(idx, ql, s);
        else if (kr <= 4)
            e = launch_overflow<4>(idx, ql, s);
        else
            e = launch_overflow<8>(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_vote_search (overflow)");
    }
    if (ql.stage_ms) {
        MRPT_CUDA_TRY(cudaEventRecord(idx->ev[3], s));
        MRPT_CUDA_TRY(cudaEventSynchronize(idx->ev[3]));
        MRPT_CUDA_TRY(cudaEventElapsedTime(&ql.stage_ms[0], idx->ev[0], idx->ev[1]));
        MRPT_CUDA_TRY(cudaEventElapsedTime(&ql.stage_ms[1], idx->ev[1], idx->ev[2]));
        MRPT_CUDA_TRY(cudaEventElapsedTime(&ql.stage_ms[2], idx->ev[2], idx->ev[3]));
        MRPT_CUDA_TRY(cudaEventElapsedTime(&ql.stage_ms[3], idx->ev[0], idx->ev[3]));
    }
    return MRPT_OK;
}

}  // namespace mrpt

namespace mrpt {

// The same two kernels as launch_query, with the leaf-of-query table in
// ql.leaf and the work counter at `work`, both supplied by the caller; no
// stage timing.  Used by the allocation-free entry point.
int launch_query_with_counter(mrpt_index *idx, const QueryLaunch &ql, uint32_t *work) {
    cudaStream_t s = idx->stream;
    if (ql.m == 0) return MRPT_OK;
    const int64_t per_q = int64_t(idx->d) * 4;
    cudaError_t e;
    if (per_q * 32 <= 110 * 1024)
        e = launch_route<32>(idx, ql, s);
    else if (per_q * 16 <= 110 * 1024)
        e = launch_route<16>(idx, ql, s);
    else if (per_q * 8 <= 160 * 1024)
        e = launch_route<8>(idx, ql, s);
    else if (per_q * 4 <= 160 * 1024)
        e = launch_route<4>(idx, ql, s);
    else if (per_q * 2 <= 200 * 1024)
        e = launch_route<2>(idx, ql, s);
    else
        e = launch_route<1>(idx, ql, s);
    if (e != cudaSuccess) return cuda_fail(e, "k_query_route");
    const int kr = (ql.k + 31) / 32;
    if (kr <= 1)
        e = launch_vote_with_counter<1>(idx, ql, s, work);
    else if (kr <= 2)
        e = launch_vote_with_counter<2>(idx, ql, s, work);
    else if (kr <= 4)
        e = launch_vote_with_counter<4>(idx, ql, s, work);
    else
        e = launch_vote_with_counter<8>(idx, ql, s, work);
    if (e != cudaSuccess) return cuda_fail(e, "k_vote_search");
    return MRPT_OK;
}

}  // namespace mrpt
