// Query phase (Sec. III, Algorithms 3-4) on sm_103a.  A batch runs
//
//   k_route_pairs   p = q^T R for every tree and level (Algorithm 3), then
//                   the descent p[level] <= split -> left, when 64 queries
//                   fit in shared memory (d <= 844): two queries per lane,
//                   a warp per tree, nonzeros streamed through a per-warp
//                   cp.async ring.
//   k_query_route   the same for larger d: a block stages up to 32 queries;
//                   one thread per (query, tree), lanes of a warp share
//                   trees.
//   k_vote_flat     (n <= 65,536) votes (Algorithm 4's loop) over the
//                   padded leaf layout: 8-bit counters in shared memory, four
//                   ids per lane per 16-byte load, one block of PTX per four
//                   votes; a point enters S (Sec. III-A) when its count
//                   reaches v and is appended to the query's candidate list.
//   k_vote_emit     the same for larger n, in chunks of 65,536 ids.
//   k_cand_knn      exact distances of the listed candidates, rows streamed
//                   into a per-warp ring by bulk copies, and the per-warp
//                   sorted top-k (knn(q, k, S) of Algorithm 4).
//   k_vote_search   the one-kernel variant (votes, then distances of the
//                   ids each warp emitted, then a merge of the warps'
//                   lists).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "mrpt_internal.cuh"

namespace mrpt {

// ------------------------------------------------------------- routing ----

// One thread per (query, tree): lane = query (QB = 32 queries per tile, or
// QB < 32 queries x 32/QB trees per warp when d is large).  Work items are
// (query tile, group of 16 * 32/QB trees, one per warp and lane group); a
// persistent block takes a contiguous range of items, so it stages a query
// tile once and walks its tree groups.  All lanes that share a tree read the
// same nonzeros as (dim, value bits) pairs, two per 16-byte broadcast load,
// and take their query's component from shared memory (odd row stride: no
// bank conflicts).  Each projection is an fmaf chain in ascending dimension
// from +0.0f, followed by the descent p <= split -> left (Algorithm 3).
template <int QB>
__host__ __device__ constexpr int route_tpi() { return 16 * (32 / QB); }

template <int QB>
__global__ void __launch_bounds__(512, 2) k_query_route(
    const float *__restrict__ Q, int64_t m, int32_t d, int32_t T_use, int32_t l, int64_t L,
    const int2 *__restrict__ rcol, const int2 *__restrict__ dv,
    const float *__restrict__ split, int32_t *__restrict__ leaf,
    float *__restrict__ proj, uint32_t *__restrict__ status, int64_t n_items,
    const QueryRecord *__restrict__ rec) {
    extern __shared__ float qs[];  // QB x (d | 1)
    const int stride = d | 1;
    if (rec != nullptr) {
        Q = rec->Q;
        m = rec->m;
        n_items = ((m + QB - 1) / QB) * ((T_use + route_tpi<QB>() - 1) / route_tpi<QB>());
    }
    constexpr int G = 32 / QB;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int qq = lane % QB;
    const int g = lane / QB;
    const float *qrow = qs + qq * stride;
    const int64_t inner = L - 1;
    const int ncols = T_use * l;
    const int groups = (T_use + route_tpi<QB>() - 1) / route_tpi<QB>();
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
        const int t_begin = grp * route_tpi<QB>();
        const int t_end = min(T_use, t_begin + route_tpi<QB>());
        for (int tb = t_begin + warp * G; tb < t_end; tb += nwarps * G) {
            const int t = tb + g;
            const bool tree_ok = t < t_end;
            const int tt = tree_ok ? t : t_begin;
            const float *sp = split + int64_t(tt) * inner;
            int64_t node = 0;
            for (int j = 0; j < l; ++j) {
                const int c = tt * l + j;
                const int2 sc = __ldg(rcol + c);
                const int4 *p4 = reinterpret_cast<const int4 *>(dv + sc.x);
                float acc = 0.0f;
                int k = 0;
                for (; k + 4 <= sc.y; k += 4) {
                    const int4 A = __ldg(p4 + (k >> 1)), B = __ldg(p4 + (k >> 1) + 1);
                    const float x0 = qrow[A.x], x1 = qrow[A.z], x2 = qrow[B.x], x3 = qrow[B.z];
                    acc = __fmaf_rn(x0, __int_as_float(A.y), acc);
                    acc = __fmaf_rn(x1, __int_as_float(A.w), acc);
                    acc = __fmaf_rn(x2, __int_as_float(B.y), acc);
                    acc = __fmaf_rn(x3, __int_as_float(B.w), acc);
                }
                if (k + 2 <= sc.y) {
                    const int4 A = __ldg(p4 + (k >> 1));
                    acc = __fmaf_rn(qrow[A.x], __int_as_float(A.y), acc);
                    acc = __fmaf_rn(qrow[A.z], __int_as_float(A.w), acc);
                    k += 2;
                }
                if (k < sc.y) {
                    const int2 P = __ldg(dv + sc.x + k);
                    acc = __fmaf_rn(qrow[P.x], __int_as_float(P.y), acc);
                }
                if (proj != nullptr && live && tree_ok) proj[(q0 + qq) * ncols + c] = acc;
                node = 2 * node + 1 + (acc > __ldg(sp + node) ? 1 : 0);
            }
            if (live && tree_ok) leaf[(q0 + qq) * T_use + t] = int32_t(node - inner);
        }
    }
}

// Routing with two queries per lane, for d small enough that a 64-query
// tile fits in shared memory dimension-major (xs[dim][64]): one 8-byte load
// gives a lane both of its queries' components, so every nonzero read feeds
// 64 fmaf chains.  A unit is (64-query tile, tree); a persistent block of NW
// warps takes a contiguous unit range, stages each tile once and its warps
// take the tile's trees in turn.  Each warp streams its tree's nonzero pairs
// through a two-slot ring in shared memory, CH pairs per slot (one 16-byte
// cp.async per lane), the next chunk (or the next tree's first) in flight
// while the current one is read.  The split value of the next level is loaded before the column's
// chain runs.  Arithmetic per (query, column) is the same fmaf chain in
// ascending dimension from +0.0f as k_query_route (Algorithm 3).
constexpr int RP_QT = 64;  // queries per tile (two per lane)

__host__ __device__ constexpr size_t route_pairs_smem(int d, int nw, int ch) {
    return size_t(d) * RP_QT * sizeof(float) + size_t(nw) * 2 * ch * sizeof(int2);
}

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int NW, int CH>
__global__ void __launch_bounds__(NW * 32, 1) k_route_pairs(
    const float *__restrict__ Q, int64_t m, int32_t d, int32_t T_use, int32_t l, int64_t L,
    const int2 *__restrict__ rcol, const int2 *__restrict__ dv, const float *__restrict__ split,
    int32_t *__restrict__ leaf, float *__restrict__ proj, uint32_t *__restrict__ status,
    const QueryRecord *__restrict__ rec) {
    static_assert(CH % 2 == 0 && CH <= 64, "a chunk is at most one 16-byte copy per lane");
    extern __shared__ __align__(16) float xs[];  // d x RP_QT, then NW x 2 x CH pairs
    if (rec != nullptr) {
        Q = rec->Q;
        m = rec->m;
    }
    constexpr int NT = NW * 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int32_t inner = int32_t(L - 1);
    const int ncols = T_use * l;
    const int64_t n_units = ((m + RP_QT - 1) / RP_QT) * int64_t(T_use);
    const int64_t per = n_units / gridDim.x, extra = n_units % gridDim.x;
    const int64_t bx = blockIdx.x;
    int64_t u = bx * per + (bx < extra ? bx : extra);
    const int64_t u1 = u + per + (bx < extra ? 1 : 0);
    const bool vec = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0;
    const float2 *xs2 = reinterpret_cast<const float2 *>(xs) + lane;  // this lane's two queries
    int2 *ring = reinterpret_cast<int2 *>(xs + size_t(d) * RP_QT) + warp * 2 * CH;
    const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));

    // ring state (warp-uniform): slot `cur` holds pairs [cur_lo, cur_lo + CH)
    // (none at first); the other slot receives nxt_lo (-1: nothing in flight)
    int cur = 1, cur_lo = -(1 << 30), nxt_lo = -1;
    // pairs past `hi` (the end of the tree's columns) are zero-filled, never read
    auto fetch = [&](int slot, int lo, int hi) {
        const int p = lo + 2 * lane;
        const bool ok = p + 2 <= hi;
        if (2 * lane < CH)
            cp_async16_zfill(ring_s + uint32_t((slot * CH + 2 * lane) * sizeof(int2)), ok ? dv + p : dv,
                             ok ? 16u : 0u);
        cp_async_commit();
    };

    while (u < u1) {
        const int64_t tile = u / T_use;
        const int t_a = int(u - tile * T_use);
        const int64_t t_end = int64_t(t_a) + (u1 - u);
        const int t_b = t_end < int64_t(T_use) ? int(t_end) : T_use;
        const int64_t q0 = tile * RP_QT;
        // ---- stage the tile dimension-major; a query past m reads as zeros
        __syncthreads();  // the previous tile is no longer read
        {
            const int qi = tid & (RP_QT - 1);
            const int64_t row = q0 + qi;
            const bool live = row < m;
            const float *src = Q + (live ? row : 0) * int64_t(d);
            bool bad = false;
            if (vec) {
                for (int c4 = tid / RP_QT; c4 < (d >> 2); c4 += NT / RP_QT) {
                    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (live) x = __ldg(reinterpret_cast<const float4 *>(src) + c4);
                    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
                    xs[(4 * c4 + 0) * RP_QT + qi] = x.x;
                    xs[(4 * c4 + 1) * RP_QT + qi] = x.y;
                    xs[(4 * c4 + 2) * RP_QT + qi] = x.z;
                    xs[(4 * c4 + 3) * RP_QT + qi] = x.w;
                }
            } else {
                for (int c = tid / RP_QT; c < d; c += NT / RP_QT) {
                    const float x = live ? __ldg(src + c) : 0.f;
                    bad |= !isfinite(x);
                    xs[c * RP_QT + qi] = x;
                }
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, STATUS_NONFINITE_QUERY);
        }
        __syncthreads();
        const int64_t qa = q0 + 2 * lane, qb = qa + 1;
        const bool live_a = qa < m, live_b = qb < m;
        for (int t = t_a + warp; t < t_b; t += NW) {
            const int2 *rc = rcol + int64_t(t) * l;
            const int base = __ldg(&rc[0].x);
            const int2 last = __ldg(rc + (l - 1));
            const int hi = last.x + ((last.y + 1) & ~1);  // even end of the tree's pairs
            const int tn = t + NW;                        // this warp's next tree in the tile
            const float *sp = split + int64_t(t) * inner;
            // a chunk fetched for an earlier tree is zero-filled past that
            // tree's pairs: every tree reads only chunks fetched for it
            cur_lo = -(1 << 30);
            int32_t node_a = 0, node_b = 0;
            for (int j = 0; j < l; ++j) {
                const int2 sc = __ldg(rc + j);
                const float s_a = __ldg(sp + node_a), s_b = __ldg(sp + node_b);
                float acc_a = 0.0f, acc_b = 0.0f;
                int pos = sc.x;
                const int cend = sc.x + sc.y;
                while (pos < cend) {
                    if (pos < cur_lo || pos >= cur_lo + CH) {
                        // make the chunk holding `pos` current
                        const int lo = base + ((pos - base) / CH) * CH;
                        if (nxt_lo != lo) {
                            cp_async_wait_all();  // the other slot's copy (if any) is done
                            __syncwarp();
                            fetch(cur ^ 1, lo, hi);
                        }
                        cp_async_wait_all();
                        __syncwarp();
                        cur ^= 1;
                        cur_lo = lo;
                        nxt_lo = -1;
                        // prefetch the next chunk of this tree, else the next tree's first
                        if (lo + CH < hi) {
                            nxt_lo = lo + CH;
                            fetch(cur ^ 1, nxt_lo, hi);
                        } else if (tn < t_b) {
                            const int2 *rn = rcol + int64_t(tn) * l;
                            const int2 nl = __ldg(rn + (l - 1));
                            const int nb = __ldg(&rn[0].x), nhi = nl.x + ((nl.y + 1) & ~1);
                            if (nb < nhi) {
                                nxt_lo = nb;
                                fetch(cur ^ 1, nb, nhi);
                            }
                        }
                    }
                    const int lim = min(cend, cur_lo + CH);
                    const int2 *rs = ring + cur * CH - cur_lo;  // indexed by pair position
#pragma unroll 2
                    for (; pos + 4 <= lim; pos += 4) {
                        const int4 A = *reinterpret_cast<const int4 *>(rs + pos);
                        const int4 B = *reinterpret_cast<const int4 *>(rs + pos + 2);
                        const float2 x0 = xs2[A.x * (RP_QT / 2)], x1 = xs2[A.z * (RP_QT / 2)];
                        const float2 x2 = xs2[B.x * (RP_QT / 2)], x3 = xs2[B.z * (RP_QT / 2)];
                        acc_a = __fmaf_rn(x0.x, __int_as_float(A.y), acc_a);
                        acc_b = __fmaf_rn(x0.y, __int_as_float(A.y), acc_b);
                        acc_a = __fmaf_rn(x1.x, __int_as_float(A.w), acc_a);
                        acc_b = __fmaf_rn(x1.y, __int_as_float(A.w), acc_b);
                        acc_a = __fmaf_rn(x2.x, __int_as_float(B.y), acc_a);
                        acc_b = __fmaf_rn(x2.y, __int_as_float(B.y), acc_b);
                        acc_a = __fmaf_rn(x3.x, __int_as_float(B.w), acc_a);
                        acc_b = __fmaf_rn(x3.y, __int_as_float(B.w), acc_b);
                    }
                    if (pos + 2 <= lim) {
                        const int4 A = *reinterpret_cast<const int4 *>(rs + pos);
                        const float2 x0 = xs2[A.x * (RP_QT / 2)], x1 = xs2[A.z * (RP_QT / 2)];
                        acc_a = __fmaf_rn(x0.x, __int_as_float(A.y), acc_a);
                        acc_b = __fmaf_rn(x0.y, __int_as_float(A.y), acc_b);
                        acc_a = __fmaf_rn(x1.x, __int_as_float(A.w), acc_a);
                        acc_b = __fmaf_rn(x1.y, __int_as_float(A.w), acc_b);
                        pos += 2;
                    }
                    if (pos < lim) {  // the odd last pair of the column
                        const int2 P = rs[pos];
                        const float2 x0 = xs2[P.x * (RP_QT / 2)];
                        acc_a = __fmaf_rn(x0.x, __int_as_float(P.y), acc_a);
                        acc_b = __fmaf_rn(x0.y, __int_as_float(P.y), acc_b);
                        pos += 1;
                    }
                }
                if (proj != nullptr) {
                    const int c = t * l + j;
                    if (live_a) proj[qa * ncols + c] = acc_a;
                    if (live_b) proj[qb * ncols + c] = acc_b;
                }
                node_a = 2 * node_a + 1 + (acc_a > s_a ? 1 : 0);
                node_b = 2 * node_b + 1 + (acc_b > s_b ? 1 : 0);
            }
            if (live_a) leaf[qa * T_use + t] = node_a - inner;
            if (live_b) leaf[qb * T_use + t] = node_b - inner;
        }
        u += t_b - t_a;
    }
    cp_async_wait_all();  // no copy into shared memory outlives the block
}

// ---------------------------------------------------------- vote search ----

constexpr int VS_THREADS = 256;
constexpr int VS_WARPS = VS_THREADS / 32;
constexpr int CH_WORDS = 16384;          // 64 KB: 8-bit counters for 65,536 ids
constexpr int64_t CH_IDS = int64_t(CH_WORDS) * 4;
static_assert(CH_IDS == VOTE_CHUNK_IDS, "one id chunk per counter array");
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

// acc + (q - x)^2 per component, as packed two-lane float32 instructions
// (each lane rounds exactly as the scalar __fadd_rn / __fmaf_rn would).
__device__ __forceinline__ float2 sq_acc2(float2 q, float2 x, float2 acc) {
    const float2 t = __fadd2_rn(q, make_float2(-x.x, -x.y));
    return __ffma2_rn(t, t, acc);
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

// ---- TMA bulk copies (global -> shared) completed on an mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory atomic add at a 32-bit shared address; returns the old word.
__device__ __forceinline__ uint32_t atom_add_shared_u32(uint32_t addr, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v) : "memory");
    return old;
}

// One lane's share of a vote window: four leaf entries e.x..e.w at
// positions rel..rel+3 of a segment of length len.  Each entry in the
// segment adds one vote to its 8-bit counter (the byte (id - c0) & 3 of word
// (id - c0) >> 2 at shared address cnt_s); an entry outside the segment goes
// to the lane's spare word instead.  Returns a bit per entry whose count went
// from v-1 to v.  Written as one PTX block so that each step is one integer
// instruction and all four atomics are in flight together.
__device__ __forceinline__ uint32_t vote4(uint32_t cnt_s, int4 e, int32_t rel, int32_t len,
                                          int32_t c0, uint32_t spare, uint32_t vm1) {
    uint32_t emask;
    asm volatile(
        "{\n\t"
        ".reg .pred p<4>, h<4>;\n\t"
        ".reg .b32 t<4>, o<4>, s<4>, n<4>, r<4>, z, one;\n\t"
        "mov.b32 z, 0;\n\t"
        "mov.b32 one, 1;\n\t"
        "setp.lt.u32 p0, %6, %7;\n\t"
        "add.u32 t1, %6, 1;\n\t"
        "setp.lt.u32 p1, t1, %7;\n\t"
        "add.u32 t2, %6, 2;\n\t"
        "setp.lt.u32 p2, t2, %7;\n\t"
        "add.u32 t3, %6, 3;\n\t"
        "setp.lt.u32 p3, t3, %7;\n\t"
        "sub.u32 o0, %2, %8;\n\t"
        "sub.u32 o1, %3, %8;\n\t"
        "sub.u32 o2, %4, %8;\n\t"
        "sub.u32 o3, %5, %8;\n\t"
        "selp.b32 o0, o0, %9, p0;\n\t"
        "selp.b32 o1, o1, %9, p1;\n\t"
        "selp.b32 o2, o2, %9, p2;\n\t"
        "selp.b32 o3, o3, %9, p3;\n\t"
        "shl.b32 s0, o0, 3;\n\t"
        "shl.b32 s1, o1, 3;\n\t"
        "shl.b32 s2, o2, 3;\n\t"
        "shl.b32 s3, o3, 3;\n\t"
        "shf.l.wrap.b32 n0, z, one, s0;\n\t"
        "shf.l.wrap.b32 n1, z, one, s1;\n\t"
        "shf.l.wrap.b32 n2, z, one, s2;\n\t"
        "shf.l.wrap.b32 n3, z, one, s3;\n\t"
        "and.b32 t0, o0, 0xfffffffc;\n\t"
        "and.b32 t1, o1, 0xfffffffc;\n\t"
        "and.b32 t2, o2, 0xfffffffc;\n\t"
        "and.b32 t3, o3, 0xfffffffc;\n\t"
        "add.u32 t0, t0, %1;\n\t"
        "add.u32 t1, t1, %1;\n\t"
        "add.u32 t2, t2, %1;\n\t"
        "add.u32 t3, t3, %1;\n\t"
        "atom.shared.add.u32 r0, [t0], n0;\n\t"
        "atom.shared.add.u32 r1, [t1], n1;\n\t"
        "atom.shared.add.u32 r2, [t2], n2;\n\t"
        "atom.shared.add.u32 r3, [t3], n3;\n\t"
        "shf.r.wrap.b32 r0, r0, z, s0;\n\t"
        "shf.r.wrap.b32 r1, r1, z, s1;\n\t"
        "shf.r.wrap.b32 r2, r2, z, s2;\n\t"
        "shf.r.wrap.b32 r3, r3, z, s3;\n\t"
        "and.b32 r0, r0, 255;\n\t"
        "and.b32 r1, r1, 255;\n\t"
        "and.b32 r2, r2, 255;\n\t"
        "and.b32 r3, r3, 255;\n\t"
        "setp.eq.and.u32 h0, r0, %10, p0;\n\t"
        "setp.eq.and.u32 h1, r1, %10, p1;\n\t"
        "setp.eq.and.u32 h2, r2, %10, p2;\n\t"
        "setp.eq.and.u32 h3, r3, %10, p3;\n\t"
        "selp.b32 %0, 1, 0, h0;\n\t"
        "selp.b32 t1, 2, 0, h1;\n\t"
        "selp.b32 t2, 4, 0, h2;\n\t"
        "selp.b32 t3, 8, 0, h3;\n\t"
        "or.b32 %0, %0, t1;\n\t"
        "or.b32 t2, t2, t3;\n\t"
        "or.b32 %0, %0, t2;\n\t"
        "}"
        : "=r"(emask)
        : "r"(cnt_s), "r"(e.x), "r"(e.y), "r"(e.z), "r"(e.w), "r"(rel), "r"(len), "r"(c0), "r"(spare),
          "r"(vm1)
        : "memory");
    return emask;
}

// 16-byte read-only load issued only when ok != 0 (no branch); when ok == 0
// the result is unspecified and must not be used.
__device__ __forceinline__ int4 ldg4_if(const int4 *p, uint32_t ok) {
    int4 v;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %5, 0;\n\t"
        "@q ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "r"(ok));
    return v;
}

// The same for four ids that need no range check (a lane either has four
// entries of one padded leaf or none): ok == 0 sends the lane's four votes to
// its own spare word at shared address spare (no branch; results ignored).
// Counter byte id & 3 of word id >> 2 at cnt_s.
__device__ __forceinline__ uint32_t vote4p(uint32_t cnt_s, int4 e, uint32_t ok, uint32_t spare,
                                           uint32_t vm1) {
    uint32_t emask;
    asm volatile(
        "{\n\t"
        ".reg .pred p, h<4>;\n\t"
        ".reg .b32 t<4>, s<4>, n<4>, r<4>, z, one;\n\t"
        "setp.ne.u32 p, %5, 0;\n\t"
        "mov.b32 z, 0;\n\t"
        "mov.b32 one, 1;\n\t"
        "shl.b32 s0, %1, 3;\n\t"
        "shl.b32 s1, %2, 3;\n\t"
        "shl.b32 s2, %3, 3;\n\t"
        "shl.b32 s3, %4, 3;\n\t"
        "shf.l.wrap.b32 n0, z, one, s0;\n\t"
        "shf.l.wrap.b32 n1, z, one, s1;\n\t"
        "shf.l.wrap.b32 n2, z, one, s2;\n\t"
        "shf.l.wrap.b32 n3, z, one, s3;\n\t"
        "and.b32 t0, %1, 0xfffffffc;\n\t"
        "and.b32 t1, %2, 0xfffffffc;\n\t"
        "and.b32 t2, %3, 0xfffffffc;\n\t"
        "and.b32 t3, %4, 0xfffffffc;\n\t"
        "add.u32 t0, t0, %6;\n\t"
        "add.u32 t1, t1, %6;\n\t"
        "add.u32 t2, t2, %6;\n\t"
        "add.u32 t3, t3, %6;\n\t"
        "selp.b32 t0, t0, %7, p;\n\t"
        "selp.b32 t1, t1, %7, p;\n\t"
        "selp.b32 t2, t2, %7, p;\n\t"
        "selp.b32 t3, t3, %7, p;\n\t"
        "atom.shared.add.u32 r0, [t0], n0;\n\t"
        "atom.shared.add.u32 r1, [t1], n1;\n\t"
        "atom.shared.add.u32 r2, [t2], n2;\n\t"
        "atom.shared.add.u32 r3, [t3], n3;\n\t"
        "shf.r.wrap.b32 r0, r0, z, s0;\n\t"
        "shf.r.wrap.b32 r1, r1, z, s1;\n\t"
        "shf.r.wrap.b32 r2, r2, z, s2;\n\t"
        "shf.r.wrap.b32 r3, r3, z, s3;\n\t"
        "and.b32 r0, r0, 255;\n\t"
        "and.b32 r1, r1, 255;\n\t"
        "and.b32 r2, r2, 255;\n\t"
        "and.b32 r3, r3, 255;\n\t"
        "setp.eq.and.u32 h0, r0, %8, p;\n\t"
        "setp.eq.and.u32 h1, r1, %8, p;\n\t"
        "setp.eq.and.u32 h2, r2, %8, p;\n\t"
        "setp.eq.and.u32 h3, r3, %8, p;\n\t"
        "selp.b32 %0, 1, 0, h0;\n\t"
        "selp.b32 t1, 2, 0, h1;\n\t"
        "selp.b32 t2, 4, 0, h2;\n\t"
        "selp.b32 t3, 8, 0, h3;\n\t"
        "or.b32 %0, %0, t1;\n\t"
        "or.b32 t2, t2, t3;\n\t"
        "or.b32 %0, %0, t2;\n\t"
        "}"
        : "=r"(emask)
        : "r"(e.x), "r"(e.y), "r"(e.z), "r"(e.w), "r"(ok), "r"(cnt_s), "r"(spare), "r"(vm1)
        : "memory");
    return emask;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// One arrival that also announces `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it ran out.
constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 21;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = MBAR_SPIN_LIMIT) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Squared distance between the staged query and a row staged in shared
// memory (consecutive float4 per lane: no bank conflicts).
__device__ __forceinline__ float smem_row_sq_dist(const float4 *row, const float4 *q4, int nv4,
                                                  int lane) {
    float2 a = make_float2(0.f, 0.f);  // (x and z terms, y and w terms)
    for (int j = lane; j < nv4; j += 32) {
        const float4 x = row[j];
        const float4 q = q4[j];
        a = sq_acc2(make_float2(q.x, q.y), make_float2(x.x, x.y), a);
        a = sq_acc2(make_float2(q.z, q.w), make_float2(x.z, x.w), a);
    }
    return warp_sum(a.x + a.y);
}

// Two staged rows against the staged query at once: one query load feeds
// both rows and the two warp reductions interleave.  ROW is float4 (float32
// rows) or uint2 (four bfloat16 values); either way step j covers query
// components 4j .. 4j+3, so every lane reads consecutive 16-byte query
// chunks (no bank conflicts).
template <typename ROW>
__device__ __forceinline__ float4 row_chunk(const ROW &x);

template <>
__device__ __forceinline__ float4 row_chunk<float4>(const float4 &x) {
    return x;
}

template <>
__device__ __forceinline__ float4 row_chunk<uint2>(const uint2 &x) {
    return make_float4(__uint_as_float(x.x << 16), __uint_as_float(x.x & 0xffff0000u),
                       __uint_as_float(x.y << 16), __uint_as_float(x.y & 0xffff0000u));
}

template <typename ROW>
__device__ __forceinline__ void smem_rows2_sq_dist(const ROW *r0, const ROW *r1, const float4 *q4,
                                                   int nv4, int lane, float &d0, float &d1) {
    // per row: (x and z terms, y and w terms)
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int j = lane; j < nv4; j += 32) {
        const float4 q = q4[j];
        const float4 x = row_chunk<ROW>(r0[j]);
        const float4 y = row_chunk<ROW>(r1[j]);
        const float2 qlo = make_float2(q.x, q.y), qhi = make_float2(q.z, q.w);
        a = sq_acc2(qlo, make_float2(x.x, x.y), a);
        b = sq_acc2(qlo, make_float2(y.x, y.y), b);
        a = sq_acc2(qhi, make_float2(x.z, x.w), a);
        b = sq_acc2(qhi, make_float2(y.z, y.w), b);
    }
    float sa = a.x + a.y, sb = b.x + b.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    d0 = sa;
    d1 = sb;
}

// Four e4m3 values (one 32-bit word) widened to float.
__device__ __forceinline__ float4 e4m3x4_to_float4(uint32_t w) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(w & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(w >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Two staged e4m3 rows (each value times its row's scale) against the
// staged query; step j covers components 4j .. 4j+3.
__device__ __forceinline__ void smem_rows2_sq_dist_fp8(const uint32_t *r0, const uint32_t *r1,
                                                       float s0, float s1, const float4 *q4, int nv4,
                                                       int lane, float &d0, float &d1) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    const float2 ns0 = make_float2(-s0, -s0), ns1 = make_float2(-s1, -s1);
#pragma unroll 2
    for (int j = lane; j < nv4; j += 32) {
        const float4 q = q4[j];
        const float4 x = e4m3x4_to_float4(r0[j]);
        const float4 y = e4m3x4_to_float4(r1[j]);
        const float2 qlo = make_float2(q.x, q.y), qhi = make_float2(q.z, q.w);
        float2 t;
        t = __ffma2_rn(ns0, make_float2(x.x, x.y), qlo);
        a = __ffma2_rn(t, t, a);
        t = __ffma2_rn(ns1, make_float2(y.x, y.y), qlo);
        b = __ffma2_rn(t, t, b);
        t = __ffma2_rn(ns0, make_float2(x.z, x.w), qhi);
        a = __ffma2_rn(t, t, a);
        t = __ffma2_rn(ns1, make_float2(y.z, y.w), qhi);
        b = __ffma2_rn(t, t, b);
    }
    float sa = a.x + a.y, sb = b.x + b.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    d0 = sa;
    d1 = sb;
}

// float32 rows -> e4m3 rows with a per-row scale max|x| / 448 (one warp per
// row).  Row layout: row_bytes - 16 e4m3 values (zero beyond d), then the
// float32 scale, then padding.
__global__ void k_to_fp8(const float *__restrict__ X, int64_t n, int32_t dpad,
                         unsigned char *__restrict__ Y, int32_t row_bytes) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int vals = row_bytes - 16;
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const float *x = X + r * dpad;
        float mx = 0.f;
        for (int i = lane; i < dpad; i += 32) mx = fmaxf(mx, fabsf(x[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float scale = mx > 0.f ? mx / 448.0f : 1.0f;
        const float inv = 1.0f / scale;
        unsigned char *y = Y + r * row_bytes;
        for (int i = lane; i < vals; i += 32) {
            const __nv_fp8_e4m3 v(i < dpad ? x[i] * inv : 0.0f);
            y[i] = *reinterpret_cast<const unsigned char *>(&v);
        }
        if (lane == 0) *reinterpret_cast<float *>(y + vals) = scale;
        if (lane >= 1 && lane < 13) y[vals + 3 + lane] = 0;
    }
}

// float32 rows -> bfloat16 copy (round to nearest even), same row stride;
// *lossy is set when some value does not survive the rounding.
__global__ void k_to_bf16(const float *__restrict__ X, __nv_bfloat16 *__restrict__ Y, int64_t count,
                          uint32_t *__restrict__ lossy) {
    bool diff = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x) {
        const __nv_bfloat16 y = __float2bfloat16_rn(X[i]);
        Y[i] = y;
        diff |= __bfloat162float(y) != X[i];
    }
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(lossy, 1u);
}

// End of tree t's ids below lim = (c + 1) * CH_IDS inside the query's leaf
// lf of that tree (entries [lo, hi) of the tree's leaf_ids row, ids
// ascending): one load from the index's id-chunk bounds when it has them,
// else a binary search of the leaf.
__device__ __forceinline__ int32_t chunk_cut(const int32_t *chunk_bnd, int32_t n_chunks, int64_t L, int t,
                                             int32_t lf, int64_t c, const int32_t *leaf_ids, int64_t n,
                                             int32_t lo, int32_t hi, int64_t lim) {
    if (lim >= n) return hi;
    if (chunk_bnd != nullptr)
        return __ldg(chunk_bnd + (int64_t(t) * L + lf) * (n_chunks + 1) + (c + 1));
    const int32_t *ids = leaf_ids + int64_t(t) * n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (int64_t(__ldg(ids + mid)) < lim)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
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
    const QueryRecord *rec;      // plan mode: Q, outputs and m of the batch
    // vote layout (n <= 65,536): voted as in k_vote_flat
    const int4 *leaf4;
    const int32_t *leaf_off4;
    int64_t s4;
    int32_t sentinel;
    // n > 65,536: id-chunk bounds of every leaf (null: binary searches)
    const int32_t *chunk_bnd;
    int32_t n_chunks;
    int64_t L;
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
__global__ void __launch_bounds__(VS_THREADS, 3) k_vote_search(const VoteSearchArgs a0) {
    VoteSearchArgs a = a0;
    if (a.rec != nullptr) {
        a.Q = a.rec->Q;
        a.out_ids = a.rec->out_ids;
        a.out_dists = a.rec->out_dists;
        a.m = a.rec->m;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);                        // a.cnt_words
    float *qv = reinterpret_cast<float *>(smem + size_t(a.region_bytes));      // dpad
    int32_t *wbuf = reinterpret_cast<int32_t *>(qv + a.dpad);                  // VS_WARPS * WBUF
    int32_t *cur = wbuf + VS_WARPS * WBUF;                                      // T_use
    int32_t *lend = cur + a.T_use;                                              // T_use
    int32_t *cend = lend + a.T_use;                                             // T_use
    int32_t *lfs = cend + a.T_use;                                              // T_use: the query's leaves
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
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_total = 0ull;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;

        for (int i = tid; i < a.dpad; i += VS_THREADS) qv[i] = (i < a.d) ? a.Q[qi * a.d + i] : 0.f;
        for (int t = tid; t < a.T_use; t += VS_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * a.T_use + t];
            lfs[t] = lf;
            if (a.leaf4 != nullptr) {  // first 16-byte unit and length of the padded leaf
                cur[t] = a.leaf_off4[lf];
                lend[t] = a.leaf_off4[lf + 1] - cur[t];
            } else {
                cur[t] = a.leaf_off[lf];
                lend[t] = a.leaf_off[lf + 1];
            }
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

        if (a.leaf4 != nullptr) {
            // one id chunk, voted over the vote layout as in k_vote_flat: each
            // warp takes its trees' 128-id windows; lanes past a leaf vote
            // into their spare word; emitted ids are appended to the warp's
            // buffer in lane order
            const uint32_t cnt_s = smem_u32(cnt);
            const uint32_t spare = cnt_s + 4u * uint32_t(a.cnt_words + 4 + lane);
            {
                uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
                for (int w = tid; w < (a.cnt_words >> 2); w += VS_THREADS) c4[w] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncthreads();
            int nb = 0;
            for (int t = warp; t < a.T_use; t += VS_WARPS) {
                const int4 *lp = a.leaf4 + int64_t(t) * a.s4 + cur[t];
                const int32_t len4 = lend[t];
                for (int w0 = 0; w0 < len4; w0 += 32) {
                    const uint32_t ok = w0 + lane < len4 ? 1u : 0u;
                    const int4 q = ldg4_if(lp + w0 + lane, ok);
                    uint32_t em = vote4p(cnt_s, q, ok, spare, vm1);
                    const int32_t e4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (e4[u] == a.sentinel) em &= ~(1u << u);
                    if (__any_sync(0xffffffffu, em != 0u)) {
                        const int mine = __popc(em);
                        int incl = mine;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int y = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += y;
                        }
                        const int tot = __shfl_sync(0xffffffffu, incl, 31);
                        int pos = nb + incl - mine;
                        unsigned long long base = 0;
                        if (track) {
                            if (lane == 0) base = atomicAdd(&s_total, (unsigned long long)tot);
                            base = __shfl_sync(0xffffffffu, base, 0);
                        }
                        int64_t slot = int64_t(base) + incl - mine;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if ((em >> u) & 1u) {
                                mybuf[pos++] = e4[u];
                                if (a.dbg_cand != nullptr && slot < a.cand_cap) a.dbg_cand[qi * a.cand_cap + slot] = e4[u];
                                ++slot;
                            }
                        }
                        nb += tot;
                    }
                    if (nb >= 64) {
                        drain(nb);
                        nb = 0;
                    }
                }
            }
            if (nb > 0) drain(nb);
            __syncthreads();
            if (a.dbg_votes != nullptr) {
                for (int w = tid; w < int((a.n + 3) >> 2); w += VS_THREADS) {
                    const uint32_t word = cnt[w];
                    for (int b = 0; b < 4; ++b) {
                        const int64_t id = 4 * int64_t(w) + b;
                        if (id < a.n) a.dbg_votes[qi * a.n + id] = uint8_t((word >> (8 * b)) & 0xffu);
                    }
                }
                __syncthreads();
            }
        }
        for (int64_t c0 = 0; a.leaf4 == nullptr && c0 < a.n; c0 += CH_IDS) {
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
            for (int t = tid; t < a.T_use; t += VS_THREADS)
                cend[t] = chunk_cut(a.chunk_bnd, a.n_chunks, a.L, t, lfs[t], c0 / CH_IDS, a.leaf_ids, a.n, cur[t],
                                    lend[t], lim);
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
//   k_vote_emit  votes over 128-entry windows of the query's leaves (one
//                16-byte load per lane, windows balanced over the warps) and
//                writes each query's candidate set S to a per-query list in
//                global memory; it carries no distance state, so a block
//                has 16 warps.  A list holds T ceil(n / 2^l) / v entries,
//                the most S can have (Sec. III-B), so every query fits.
//   k_cand_knn   one warp per (query, chunk of the list) work item: exact
//                distances of the chunk's candidates and the warp's sorted
//                top-k; the item that completes a query merges the lists.

constexpr int VE_THREADS = 512;
constexpr int VE_WARPS = VE_THREADS / 32;
constexpr int VE_WIN = 128;  // leaf entries per warp window (4 per lane, one 16-byte load)

struct VoteEmitArgs {
    int64_t n;
    const int32_t *leaf_of_q;
    int32_t T_use;
    const int32_t *leaf_off;
    const int32_t *leaf_ids;
    int64_t m;
    int32_t v;
    int32_t *cand;         // m x capq candidate ids (capq >= |S| of every query)
    int32_t capq;
    int32_t *ncand;        // m: |S|
    uint32_t *work;
    int32_t cnt_words;
    uint8_t *dbg_votes;
    int64_t *dbg_ncand;
    int32_t *dbg_cand;
    int64_t cand_cap;
    int2 *items;           // (query, chunk) work items of k_cand_knn
    uint32_t *n_items;
    int32_t chunk;         // candidates per work item
    int32_t *done;         // per query: finished work items
    const QueryRecord *rec;  // plan mode: m of the batch
    // vote layout (k_vote_flat)
    const int4 *leaf4;
    const int32_t *leaf_off4;
    int64_t s4;
    int32_t win;           // 128-entry windows per leaf
    uint64_t win_magic;    // ceil(2^32 / win): i / win = (i * win_magic) >> 32 for i < 256 * win
    int32_t sentinel;
    // n > 65,536: id-chunk bounds of every leaf (null: binary searches)
    const int32_t *chunk_bnd;
    int32_t n_chunks;
    int64_t L;
};

// Called by one thread once a query's votes are all in: records |S| and
// appends the query's work items.  capq bounds |S| (|S| <= T ceil(n / 2^l) / v,
// Sec. III-B), so the list always held every candidate.
__device__ __forceinline__ void publish_items(const VoteEmitArgs &a, int64_t qi, int c) {
    a.ncand[qi] = c;
    if (a.dbg_ncand != nullptr) a.dbg_ncand[qi] = c;
    const int cc = min(c, a.capq);
    const int nch = item_count(cc, item_size(cc, a.chunk));
    const uint32_t b0 = atomicAdd(a.n_items, uint32_t(nch));
    for (int j = 0; j < nch; ++j) a.items[b0 + j] = make_int2(int32_t(qi), j);
    a.done[qi] = 0;
}

// Per query (one block, queries taken from an atomic counter):
//   1. the query's leaf in each tree gives one segment of that tree's leaf
//      array (ids ascending);
//   2. per id chunk: clear the 8-bit counters; cut every segment to the ids
//      of the chunk; split the segments into windows of 128 entries that
//      start on a 4-entry boundary, so a lane reads its 4 entries with one
//      16-byte load; each warp takes a contiguous run of windows (balanced
//      over the block, whatever the leaf sizes);
//   3. every valid entry adds one vote with a shared-memory atomic; the lane
//      whose increment takes a count from v-1 to v appends the id to the
//      query's list (Algorithm 4: a point enters S when its vote count
//      reaches v).  List order is not fixed; the set is.
__global__ void __launch_bounds__(VE_THREADS, 3) k_vote_emit(const VoteEmitArgs a0) {
    VoteEmitArgs a = a0;
    if (a.rec != nullptr) a.m = a.rec->m;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // cnt_words + 32 spare words
    // per tree in this chunk: int4 index of the aligned segment start, and
    // (segment length, entries before the segment in its first int4)
    int64_t *tg4 = reinterpret_cast<int64_t *>(cnt + a.cnt_words + 32);
    int2 *tlh = reinterpret_cast<int2 *>(tg4 + a.T_use);
    int32_t *cur = reinterpret_cast<int32_t *>(tlh + a.T_use);     // first entry left, per tree
    int32_t *lend = cur + a.T_use;                                  // end of the query's leaf
    int32_t *cend = lend + a.T_use;                                 // end inside this chunk
    int32_t *wpre = cend + a.T_use;                                 // T_use + 1: first window
    int32_t *lfs = wpre + a.T_use + 1;                              // T_use: the query's leaves
    __shared__ int64_t s_q;
    __shared__ int s_cnt;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint32_t vm1 = uint32_t(a.v - 1);
    const int T = a.T_use;
    int32_t next_cut = 0;  // thread t < T: tree t's cut of the next id chunk

    for (;;) {
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;
        for (int t = tid; t < T; t += VE_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * T + t];
            lfs[t] = lf;
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
            // this chunk's part of every segment and its window count (the
            // thread of tree t also wrote cur[t] and lend[t])
            const int64_t lim = c0 + CH_IDS;
            // thread t < T (T <= 255 < VE_THREADS) cuts tree t; with chunk
            // bounds it loaded this cut during the previous chunk
            if (tid < T) {
                const int t = tid;
                const int32_t p = cur[t];
                const int64_t c = c0 / CH_IDS;
                const int32_t hi = (a.chunk_bnd != nullptr && c > 0 && lim < a.n)
                                       ? next_cut
                                       : chunk_cut(a.chunk_bnd, a.n_chunks, a.L, t, lfs[t], c, a.leaf_ids, a.n, p,
                                                   lend[t], lim);
                if (a.chunk_bnd != nullptr && lim + CH_IDS < a.n)
                    next_cut = __ldg(a.chunk_bnd + (int64_t(t) * a.L + lfs[t]) * (a.n_chunks + 1) + (c + 2));
                cend[t] = hi;
                const int64_t g = int64_t(t) * a.n + p;
                const int32_t head = int32_t(g & 3);
                tg4[t] = (g - head) >> 2;
                tlh[t] = make_int2(hi - p, head);
                wpre[t] = p < hi ? (hi - p + head + VE_WIN - 1) / VE_WIN : 0;
            }
            __syncthreads();
            if (warp == 0) {  // exclusive scan of the window counts
                int run = 0;
                for (int b = 0; b < T; b += 32) {
                    const int t = b + lane;
                    const int x = t < T ? wpre[t] : 0;
                    int s = x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, s, o);
                        if (lane >= o) s += y;
                    }
                    if (t < T) wpre[t] = run + s - x;
                    run += __shfl_sync(0xffffffffu, s, 31);
                }
                if (lane == 0) wpre[T] = run;
            }
            __syncthreads();
            // this warp's windows [i0, i1)
            const int W = wpre[T];
            const int i0 = int((int64_t(W) * warp) / VE_WARPS);
            const int i1 = int((int64_t(W) * (warp + 1)) / VE_WARPS);
            int t = 0;
            {
                int hi = T;  // last tree whose first window is <= i0
                while (hi - t > 1) {
                    const int mid = (t + hi) >> 1;
                    if (wpre[mid] <= i0)
                        t = mid;
                    else
                        hi = mid;
                }
            }
            const int32_t c0i = int32_t(c0);
            // an entry outside the segment is redirected to the lane's spare
            // counter word (past the chunk's words; never read back), so the
            // vote loop has no branch per entry
            const uint32_t spare = 4u * uint32_t(a.cnt_words + lane);
            const uint32_t cnt_s = smem_u32(cnt);
            if (i0 < i1) {
                // fetch cursor: tree t, its windows [wf, wn), its segment
                // (aligned start tp, head = entries before the segment start,
                // length len)
                int wf = wpre[t], wn = wpre[t + 1];
                int32_t lrel = 0, len = 0;  // lane's first entry in the tree's first window
                const int4 *tpl = nullptr;  // the lane's int4 in the tree's first window
                auto load_tree = [&]() {
                    const int2 lh = tlh[t];
                    len = lh.x;
                    lrel = 4 * lane - lh.y;
                    tpl = reinterpret_cast<const int4 *>(a.leaf_ids) + tg4[t] + lane;
                };
                load_tree();
                // window i: the lane's 4 entries q and the first one's
                // position rel in the segment
                auto fetch = [&](int i, int32_t &rel, int32_t &ln, int4 &q) {
                    if (i >= wn) {
                        do {
                            ++t;
                            wf = wn;
                            wn = wpre[t + 1];
                        } while (i >= wn);
                        load_tree();
                    }
                    const int32_t j0 = (i - wf) * (VE_WIN / 4);
                    rel = 4 * j0 + lrel;
                    ln = len;
                    if (rel < len) q = __ldg(tpl + j0);
                };
                auto vote = [&](const int4 &q, int32_t rel, int32_t ln) {
                    const uint32_t emask = vote4(cnt_s, q, rel, ln, c0i, spare, vm1);
                    if (emask != 0u) {
                        const int32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if ((emask >> u) & 1u) {
                                const int slot = atomicAdd(&s_cnt, 1);
                                if (slot < a.capq) clist[slot] = e[u];
                                if (a.dbg_cand != nullptr && slot < a.cand_cap)
                                    a.dbg_cand[qi * a.cand_cap + slot] = e[u];
                            }
                        }
                    }
                };
                // two windows per step, each loaded one window ahead
                int32_t ra = 0, la = 0, rb = 0, lb = 0;
                int4 qa = make_int4(0, 0, 0, 0), qb = make_int4(0, 0, 0, 0);
                fetch(i0, ra, la, qa);
                int i = i0;
                for (; i + 1 < i1; i += 2) {
                    fetch(i + 1, rb, lb, qb);
                    vote(qa, ra, la);
                    if (i + 2 < i1) fetch(i + 2, ra, la, qa);
                    vote(qb, rb, lb);
                }
                if (i < i1) vote(qa, ra, la);
            }
            __syncthreads();
            for (int t2 = tid; t2 < T; t2 += VE_THREADS) cur[t2] = cend[t2];
            if (a.dbg_votes != nullptr) {
                for (int w = tid; w < nwords; w += VE_THREADS) {
                    const uint32_t word = cnt[w];
                    for (int b = 0; b < 4; ++b) {
                        const int64_t id2 = c0 + 4 * int64_t(w) + b;
                        if (id2 < a.n) a.dbg_votes[qi * a.n + id2] = uint8_t((word >> (8 * b)) & 0xffu);
                    }
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            const int c = s_cnt;
            publish_items(a, qi, c);
        }
    }
}

// k_vote_emit for leaves whose share of a chunk is short (large n, small
// leaves).  Per query (one block, queries taken from an atomic counter):
//   1. the query's leaf in each tree gives one segment of that tree's leaf
//      array (ids ascending);
//   2. per id chunk: clear the 8-bit counters; cut every segment to the ids
//      of the chunk (a binary search per tree); lay the cut segments end to
//      end and split that flat list into windows of 128 entries, so windows
//      stay full however short each tree's share of a chunk is; warps take
//      contiguous runs of windows;
//   3. a lane finds the tree of its four entries by a binary search over the
//      segments' starts, loads the ids and votes them (vote4); the lane whose
//      increment takes a count from v-1 to v appends the id to the query's
//      list (Algorithm 4: a point enters S when its count reaches v).  List
//      order is not fixed; the set is.
__global__ void __launch_bounds__(VE_THREADS, 3) k_vote_packed(const VoteEmitArgs a0) {
    VoteEmitArgs a = a0;
    if (a.rec != nullptr) a.m = a.rec->m;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);  // cnt_words + 32 spare words
    int32_t *cur = reinterpret_cast<int32_t *>(cnt + a.cnt_words + 32);  // first entry left, per tree
    int32_t *lend = cur + a.T_use;                                  // end of the query's leaf
    int32_t *cend = lend + a.T_use;                                 // end inside this chunk
    int32_t *fpre = cend + a.T_use;                                 // T_use + 1: flat start of each cut segment
    int32_t *lfs = fpre + a.T_use + 1;                              // T_use: the query's leaves
    __shared__ int64_t s_q;
    __shared__ int s_cnt;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint32_t vm1 = uint32_t(a.v - 1);
    const int T = a.T_use;
    int32_t next_cut = 0;  // thread t < T: tree t's cut of the next id chunk
    const uint32_t cnt_s = smem_u32(cnt);
    const uint32_t spare = 4u * uint32_t(a.cnt_words + lane);

    for (;;) {
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;
        for (int t = tid; t < T; t += VE_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * T + t];
            lfs[t] = lf;
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
            // this chunk's part of every segment (the thread of tree t also
            // wrote cur[t] and lend[t])
            const int64_t lim = c0 + CH_IDS;
            // thread t < T (T <= 255 < VE_THREADS) cuts tree t; with chunk
            // bounds it loaded this cut during the previous chunk
            if (tid < T) {
                const int t = tid;
                const int32_t p = cur[t];
                const int64_t c = c0 / CH_IDS;
                const int32_t hi = (a.chunk_bnd != nullptr && c > 0 && lim < a.n)
                                       ? next_cut
                                       : chunk_cut(a.chunk_bnd, a.n_chunks, a.L, t, lfs[t], c, a.leaf_ids, a.n, p,
                                                   lend[t], lim);
                if (a.chunk_bnd != nullptr && lim + CH_IDS < a.n)
                    next_cut = __ldg(a.chunk_bnd + (int64_t(t) * a.L + lfs[t]) * (a.n_chunks + 1) + (c + 2));
                cend[t] = hi;
                fpre[t] = hi - p;
            }
            __syncthreads();
            if (warp == 0) {  // exclusive scan of the cut lengths
                int run = 0;
                for (int b = 0; b < T; b += 32) {
                    const int t = b + lane;
                    const int x = t < T ? fpre[t] : 0;
                    int s = x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, s, o);
                        if (lane >= o) s += y;
                    }
                    if (t < T) fpre[t] = run + s - x;
                    run += __shfl_sync(0xffffffffu, s, 31);
                }
                if (lane == 0) fpre[T] = run;
            }
            __syncthreads();
            const int F = fpre[T];
            const int W = (F + VE_WIN - 1) / VE_WIN;
            const int i0 = int((int64_t(W) * warp) / VE_WARPS);
            const int i1 = int((int64_t(W) * (warp + 1)) / VE_WARPS);
            const int32_t c0i = int32_t(c0);
            for (int i = i0; i < i1; ++i) {
                const int32_t f0 = i * VE_WIN + 4 * lane;  // the lane's first flat entry
                int32_t e[4] = {0, 0, 0, 0};
                if (f0 < F) {
                    int t = 0, hi = T;  // last tree whose cut segment starts at or before f0
                    while (hi - t > 1) {
                        const int mid = (t + hi) >> 1;
                        if (fpre[mid] <= f0)
                            t = mid;
                        else
                            hi = mid;
                    }
                    int32_t tn = fpre[t + 1];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int32_t f = f0 + u;
                        if (f < F) {
                            while (f >= tn) tn = fpre[++t + 1];
                            e[u] = __ldg(a.leaf_ids + int64_t(t) * a.n + cur[t] + (f - fpre[t]));
                        }
                    }
                }
                const uint32_t emask = vote4(cnt_s, make_int4(e[0], e[1], e[2], e[3]), f0, F, c0i,
                                             spare, vm1);
                if (emask != 0u) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if ((emask >> u) & 1u) {
                            const int slot = atomicAdd(&s_cnt, 1);
                            if (slot < a.capq) clist[slot] = e[u];
                            if (a.dbg_cand != nullptr && slot < a.cand_cap)
                                a.dbg_cand[qi * a.cand_cap + slot] = e[u];
                        }
                    }
                }
            }
            __syncthreads();
            for (int t2 = tid; t2 < T; t2 += VE_THREADS) cur[t2] = cend[t2];
            if (a.dbg_votes != nullptr) {
                for (int w = tid; w < nwords; w += VE_THREADS) {
                    const uint32_t word = cnt[w];
                    for (int b = 0; b < 4; ++b) {
                        const int64_t id2 = c0 + 4 * int64_t(w) + b;
                        if (id2 < a.n) a.dbg_votes[qi * a.n + id2] = uint8_t((word >> (8 * b)) & 0xffu);
                    }
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            const int c = s_cnt;
            publish_items(a, qi, c);
        }
    }
}

// Hashed vote counters, on request (mrpt_query_opts.vote_table; every
// query's T leaves must hold at most 3/4 VH_SLOTS entries): one pass per
// query, no id chunks.  The
// table is VH_SLOTS 32-bit words in shared memory, a word (id + 1) << 8 |
// count, 0 when empty; an id's slot is found by a multiplicative hash and
// linear probing.  The T leaves hold at most 3/4 VH_SLOTS entries, so at
// most that many distinct ids: the table never fills.  An id claims an empty
// slot with a compare-and-swap (count 1); a later vote adds 1 to the word, and
// the old count tells when it went from v - 1 to v (Algorithm 4: the id
// enters S).  T <= 255 votes fit the 8-bit count.
constexpr int VH_LOG = 15;
constexpr int VH_SLOTS = 1 << VH_LOG;  // 128 KB of shared memory
constexpr int VH_THREADS = 1024;
constexpr int VH_WARPS = VH_THREADS / 32;

// The four entries e of one lane vote together (bit u of `valid`: entry u
// is in its segment).  In each round the pending entries read their slots,
// the empty ones are claimed with compare-and-swaps, the ones holding their
// own id get an atomic add, all issued back to back; an entry whose slot holds
// another id moves to the next slot for the next round.  Returns bit u set
// when entry u's count went from v - 1 to v.
__device__ __forceinline__ uint32_t vote_hash4(uint32_t *tab, const int32_t (&e)[4], uint32_t valid,
                                               uint32_t vm1) {
    uint32_t h[4], tg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        tg[u] = (uint32_t(e[u]) + 1u) << 8;
        h[u] = (uint32_t(e[u]) * 0x9E3779B1u) >> (32 - VH_LOG);
    }
    uint32_t pend = valid, hit = 0u;
    for (int round = 0; pend != 0u && round < VH_SLOTS; ++round) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = ((pend >> u) & 1u) ? tab[h[u]] : 1u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (((pend >> u) & 1u) && w[u] == 0u) {
                w[u] = atomicCAS(tab + h[u], 0u, tg[u] | 1u);
                if (w[u] == 0u) {
                    pend &= ~(1u << u);
                    if (vm1 == 0u) hit |= 1u << u;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (((pend >> u) & 1u) && (w[u] & 0xffffff00u) == tg[u]) {
                if ((atomicAdd(tab + h[u], 1u) & 0xffu) == vm1) hit |= 1u << u;
                pend &= ~(1u << u);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if ((pend >> u) & 1u) h[u] = (h[u] + 1u) & uint32_t(VH_SLOTS - 1);
    }
    return hit;  // every entry voted: the table holds every distinct id of the query
}

// Per query (one block of 32 warps, queries taken from an atomic counter):
// clear the table; window i (128 entries: one 16-byte load per lane from
// the leaf's 16-byte-aligned start) is window i % K of tree i / K, K the
// windows of the longest leaf (leaf sizes differ by at most one); warps take
// windows w, w + 32, ...; every entry in its tree's segment votes.
__global__ void __launch_bounds__(VH_THREADS, 1) k_vote_hash(const VoteEmitArgs a0) {
    VoteEmitArgs a = a0;
    if (a.rec != nullptr) a.m = a.rec->m;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem);           // VH_SLOTS words
    int64_t *tg4 = reinterpret_cast<int64_t *>(tab + VH_SLOTS);    // per tree: aligned int4 start
    int2 *tlh = reinterpret_cast<int2 *>(tg4 + a.T_use);           // per tree: (length, head)
    __shared__ int64_t s_q;
    __shared__ int s_cnt;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint32_t vm1 = uint32_t(a.v - 1);
    const int T = a.T_use;
    const int K = a.win;  // windows per tree
    const int W = T * K;
    for (;;) {
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_cnt = 0;
        }
        {
            uint4 *t4 = reinterpret_cast<uint4 *>(tab);
            for (int w = tid; w < VH_SLOTS / 4; w += VH_THREADS) t4[w] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        const int64_t qi = s_q;
        if (qi < 0) break;
        for (int t = tid; t < T; t += VH_THREADS) {
            const int32_t lf = a.leaf_of_q[qi * T + t];
            const int32_t p = a.leaf_off[lf], e = a.leaf_off[lf + 1];
            const int64_t g = int64_t(t) * a.n + p;
            const int32_t head = int32_t(g & 3);
            tg4[t] = (g - head) >> 2;
            tlh[t] = make_int2(e - p, head);
        }
        __syncthreads();
        int32_t *clist = a.cand + qi * int64_t(a.capq);
        for (int i = warp; i < W; i += VH_WARPS) {
            const int t = i / K;
            const int j = i - t * K;
            const int2 lh = tlh[t];
            const int32_t rel = 4 * (32 * j + lane) - lh.y;  // segment position of the lane's first entry
            const uint32_t ok = rel + 3 >= 0 && rel < lh.x;
            const int4 q = ldg4_if(reinterpret_cast<const int4 *>(a.leaf_ids) + tg4[t] + 32 * j + lane, ok);
            if (ok) {
                const int32_t e[4] = {q.x, q.y, q.z, q.w};
                uint32_t valid = 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) valid |= uint32_t(rel + u >= 0 && rel + u < lh.x) << u;
                const uint32_t hit = vote_hash4(tab, e, valid, vm1);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if ((hit >> u) & 1u) {
                        const int slot = atomicAdd(&s_cnt, 1);
                        if (slot < a.capq) clist[slot] = e[u];
                        if (a.dbg_cand != nullptr && slot < a.cand_cap) a.dbg_cand[qi * a.cand_cap + slot] = e[u];
                    }
                }
            }
        }
        __syncthreads();  // every vote of this query is in
        if (a.dbg_votes != nullptr) {
            uint8_t *row = a.dbg_votes + qi * a.n;
            for (int64_t x = tid; x < a.n; x += VH_THREADS) row[x] = 0;
            __syncthreads();
            for (int h = tid; h < VH_SLOTS; h += VH_THREADS) {
                const uint32_t w = tab[h];
                if (w != 0u) row[(w >> 8) - 1u] = uint8_t(w & 0xffu);
            }
        }
        if (tid == 0) publish_items(a, qi, s_cnt);
        __syncthreads();  // the table and s_cnt are reused by the next query
    }
}

// One lane's four entries e.x..e.w of a vote window: each adds one vote to
// its 8-bit counter (byte id & 3 of word id >> 2 at shared address cnt_s);
// with ok == 0 the four votes go to the lane's own spare word at shared
// address spare instead (a select: predicated shared atomics cost a branch
// each).  The increment 1 << 8 (id & 3) is one byte permute (prmt.b4e of
// the word 1 selected by id & 3), and so is the old count of the entry's
// byte (prmt.f4e moves byte id & 3 of the old word to byte 0).  x receives
// the four old counts, entry u in byte u, each XOR v-1: a zero byte marks an
// entry whose count went from v-1 to v (x is unspecified when ok == 0).  The
// result is nonzero when ok != 0 and x has a zero byte, tested word-wide:
// (x - 0x01010101) & ~x & 0x80808080 is nonzero iff some byte of x is zero.
__device__ __forceinline__ uint32_t vote4h(uint32_t cnt_s, int4 e, uint32_t ok, uint32_t vm1x4,
                                           uint32_t spare, uint32_t &x) {
    uint32_t hit;
    asm volatile(
        "{\n\t"
        ".reg .pred p, h;\n\t"
        ".reg .b32 t<4>, n<4>, r<4>, z, one;\n\t"
        "setp.ne.u32 p, %6, 0;\n\t"
        "mov.b32 z, 0;\n\t"
        "mov.b32 one, 1;\n\t"
        "prmt.b32.b4e n0, one, z, %2;\n\t"
        "prmt.b32.b4e n1, one, z, %3;\n\t"
        "prmt.b32.b4e n2, one, z, %4;\n\t"
        "prmt.b32.b4e n3, one, z, %5;\n\t"
        "and.b32 t0, %2, 0xfffffffc;\n\t"
        "and.b32 t1, %3, 0xfffffffc;\n\t"
        "and.b32 t2, %4, 0xfffffffc;\n\t"
        "and.b32 t3, %5, 0xfffffffc;\n\t"
        "add.u32 t0, t0, %7;\n\t"
        "add.u32 t1, t1, %7;\n\t"
        "add.u32 t2, t2, %7;\n\t"
        "add.u32 t3, t3, %7;\n\t"
        "selp.b32 t0, t0, %9, p;\n\t"
        "selp.b32 t1, t1, %9, p;\n\t"
        "selp.b32 t2, t2, %9, p;\n\t"
        "selp.b32 t3, t3, %9, p;\n\t"
        "atom.shared.add.u32 r0, [t0], n0;\n\t"
        "atom.shared.add.u32 r1, [t1], n1;\n\t"
        "atom.shared.add.u32 r2, [t2], n2;\n\t"
        "atom.shared.add.u32 r3, [t3], n3;\n\t"
        "prmt.b32.f4e r0, r0, z, %2;\n\t"
        "prmt.b32.f4e r1, r1, z, %3;\n\t"
        "prmt.b32.f4e r2, r2, z, %4;\n\t"
        "prmt.b32.f4e r3, r3, z, %5;\n\t"
        "prmt.b32 r0, r0, r1, 0x0040;\n\t"
        "prmt.b32 r2, r2, r3, 0x0040;\n\t"
        "prmt.b32 r0, r0, r2, 0x5410;\n\t"
        "xor.b32 %1, r0, %8;\n\t"
        "sub.u32 r1, %1, 0x01010101;\n\t"
        "not.b32 r2, %1;\n\t"
        "and.b32 r1, r1, r2;\n\t"
        "and.b32 r1, r1, 0x80808080;\n\t"
        "setp.ne.and.u32 h, r1, 0, p;\n\t"
        "selp.u32 %0, 1, 0, h;\n\t"
        "}"
        : "=r"(hit), "=r"(x)
        : "r"(e.x), "r"(e.y), "r"(e.z), "r"(e.w), "r"(ok), "r"(cnt_s), "r"(vm1x4), "r"(spare)
        : "memory");
    return hit;
}

// vote4h for a lane whose four entries all lie in the leaf (no spare-word
// select): the same increments, old counts and test.
__device__ __forceinline__ uint32_t vote4f(uint32_t cnt_s, int4 e, uint32_t vm1x4, uint32_t &x) {
    uint32_t hit;
    asm volatile(
        "{\n\t"
        ".reg .pred h;\n\t"
        ".reg .b32 t<4>, n<4>, r<4>, z, one;\n\t"
        "mov.b32 z, 0;\n\t"
        "mov.b32 one, 1;\n\t"
        "prmt.b32.b4e n0, one, z, %2;\n\t"
        "prmt.b32.b4e n1, one, z, %3;\n\t"
        "prmt.b32.b4e n2, one, z, %4;\n\t"
        "prmt.b32.b4e n3, one, z, %5;\n\t"
        "and.b32 t0, %2, 0xfffffffc;\n\t"
        "and.b32 t1, %3, 0xfffffffc;\n\t"
        "and.b32 t2, %4, 0xfffffffc;\n\t"
        "and.b32 t3, %5, 0xfffffffc;\n\t"
        "add.u32 t0, t0, %6;\n\t"
        "add.u32 t1, t1, %6;\n\t"
        "add.u32 t2, t2, %6;\n\t"
        "add.u32 t3, t3, %6;\n\t"
        "atom.shared.add.u32 r0, [t0], n0;\n\t"
        "atom.shared.add.u32 r1, [t1], n1;\n\t"
        "atom.shared.add.u32 r2, [t2], n2;\n\t"
        "atom.shared.add.u32 r3, [t3], n3;\n\t"
        "prmt.b32.f4e r0, r0, z, %2;\n\t"
        "prmt.b32.f4e r1, r1, z, %3;\n\t"
        "prmt.b32.f4e r2, r2, z, %4;\n\t"
        "prmt.b32.f4e r3, r3, z, %5;\n\t"
        "prmt.b32 r0, r0, r1, 0x0040;\n\t"
        "prmt.b32 r2, r2, r3, 0x0040;\n\t"
        "prmt.b32 r0, r0, r2, 0x5410;\n\t"
        "xor.b32 %1, r0, %7;\n\t"
        "sub.u32 r1, %1, 0x01010101;\n\t"
        "not.b32 r2, %1;\n\t"
        "and.b32 r1, r1, r2;\n\t"
        "and.b32 r1, r1, 0x80808080;\n\t"
        "setp.ne.u32 h, r1, 0;\n\t"
        "selp.u32 %0, 1, 0, h;\n\t"
        "}"
        : "=r"(hit), "=r"(x)
        : "r"(e.x), "r"(e.y), "r"(e.z), "r"(e.w), "r"(cnt_s), "r"(vm1x4)
        : "memory");
    return hit;
}

// k_vote_emit for an index whose ids fit one counter array (n <= 65,536),
// over the vote layout: every leaf starts on a 16-byte boundary and is padded
// with the sentinel to a multiple of 4 ids, so a lane's 16-byte load is four
// ids of one leaf (or lies past the leaf and votes nothing).  A window is 256
// entries of one leaf (two 16-byte loads per lane, 64 apart in 16-byte
// units); every leaf spans the same number a.win of windows, and window i of
// the query is window i % win of tree i / win.  Warp w takes windows w,
// w + 16, w + 32, ... two at a time (four loads in flight before any vote).
// ONE: every leaf is one window (win = 1: window i is tree i's leaf) of at
// least 32 16-byte units, so the first 32 units of every window lie in the
// leaf and vote with no range select.
template <bool ONE>
__global__ void __launch_bounds__(VE_THREADS, 3) k_vote_flat(const VoteEmitArgs a0) {
    VoteEmitArgs a = a0;
    if (a.rec != nullptr) a.m = a.rec->m;
    extern __shared__ __align__(16) unsigned char smem[];
    // cnt_words counter words, the sentinel's word (+35 unused), then per
    // tree (first 16-byte unit of the query's leaf, its 16-byte units)
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);
    int2 *seg = reinterpret_cast<int2 *>(cnt + a.cnt_words + 36);
    __shared__ int64_t s_q;
    __shared__ int s_cnt;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const uint32_t vm1x4 = uint32_t(a.v - 1) * 0x01010101u;
    const int T = a.T_use;
    const int K = a.win;
    const int W = T * K;
    const uint32_t cnt_s = smem_u32(cnt);
    const uint32_t spare = cnt_s + 4u * uint32_t(a.cnt_words + 4 + lane);

    // The next query is claimed, and its leaves looked up, while the current
    // one votes: thread t < T (T <= 255 < VE_THREADS) keeps tree t's leaf of
    // the next query in registers.
    if (tid == 0) {
        const uint32_t w = atomicAdd(a.work, 1u);
        s_q = int64_t(w) < a.m ? int64_t(w) : -1;
    }
    __syncthreads();
    int64_t qi = s_q;
    int32_t pf_o = 0, pf_e = 0;
    if (qi >= 0 && tid < T) {
        const int32_t lf = a.leaf_of_q[qi * T + tid];
        pf_o = a.leaf_off4[lf];
        pf_e = a.leaf_off4[lf + 1];
    }
    while (qi >= 0) {
        // tree t's leaf starts at 16-byte unit t * s4 + off4 (< 2^31: T s4 is
        // at most 255 (n / 4 + 2^l) for n <= 65,536)
        if (tid < T) seg[tid] = make_int2(int32_t(int64_t(tid) * a.s4) + pf_o, pf_e - pf_o);
        {
            uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
            const int n4 = a.cnt_words >> 2;
            for (int w = tid; w < n4; w += VE_THREADS) c4[w] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (tid == 0) {
            const uint32_t w = atomicAdd(a.work, 1u);
            s_q = int64_t(w) < a.m ? int64_t(w) : -1;
            s_cnt = 0;
        }
        __syncthreads();
        const int64_t qn = s_q;
        int32_t pf_lf = 0;
        if (qn >= 0 && tid < T) pf_lf = __ldg(a.leaf_of_q + qn * T + tid);
        int32_t *clist = a.cand + qi * int64_t(a.capq);
        // rare path: append the entries whose count reached v (Algorithm 4's
        // emission; the sentinel is never a candidate).  Bit 7 of byte u of
        // zb is set iff byte u of x is zero.
        auto emit = [&](const int4 &q, uint32_t x) {
            uint32_t zb = ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x | 0x7f7f7f7fu);
            while (zb != 0u) {
                const int u = (__ffs(int(zb)) - 1) >> 3;
                zb &= zb - 1u;
                const int32_t id = u == 0 ? q.x : u == 1 ? q.y : u == 2 ? q.z : q.w;
                if (id == a.sentinel) continue;
                const int slot = atomicAdd(&s_cnt, 1);
                if (slot < a.capq) clist[slot] = id;
                if (a.dbg_cand != nullptr && slot < a.cand_cap) a.dbg_cand[qi * a.cand_cap + slot] = id;
            }
        };
        for (int i = warp; i < W; i += VE_WARPS) {
            if constexpr (ONE) {
                const int2 s0 = seg[i];
                const uint32_t ok01 = lane + 32 < s0.y;
                const int4 *p0 = a.leaf4 + (s0.x + lane);
                const int4 q00 = __ldg(p0);
                const int4 q01 = ldg4_if(p0 + 32, ok01);
                uint32_t o00, o01;
                const uint32_t h0 = vote4f(cnt_s, q00, vm1x4, o00);
                const uint32_t h1 = vote4h(cnt_s, q01, ok01, vm1x4, spare, o01);
                if (__any_sync(0xffffffffu, (h0 | h1) != 0u)) {
                    if (h0) emit(q00, o00);
                    if (h1) emit(q01, o01);
                }
            } else {
                const int t0 = int((uint64_t(uint32_t(i)) * a.win_magic) >> 32);
                const int j0 = (i - t0 * K) * 64 + lane;
                const int2 s0 = seg[t0];
                const uint32_t ok00 = j0 < s0.y, ok01 = j0 + 32 < s0.y;
                const int4 *p0 = a.leaf4 + (s0.x + j0);
                const int4 q00 = ldg4_if(p0, ok00);
                const int4 q01 = ldg4_if(p0 + 32, ok01);
                uint32_t o00, o01;
                const uint32_t h0 = vote4h(cnt_s, q00, ok00, vm1x4, spare, o00);
                const uint32_t h1 = vote4h(cnt_s, q01, ok01, vm1x4, spare, o01);
                if (__any_sync(0xffffffffu, (h0 | h1) != 0u)) {
                    if (h0) emit(q00, o00);
                    if (h1) emit(q01, o01);
                }
            }
        }
        if (qn >= 0 && tid < T) {
            pf_o = __ldg(a.leaf_off4 + pf_lf);
            pf_e = __ldg(a.leaf_off4 + pf_lf + 1);
        }
        __syncthreads();  // every vote of this query is in
        if (a.dbg_votes != nullptr) {
            const int nwords = int((a.n + 3) >> 2);
            for (int w = tid; w < nwords; w += VE_THREADS) {
                const uint32_t word = cnt[w];
                for (int b = 0; b < 4; ++b) {
                    const int64_t id2 = 4 * int64_t(w) + b;
                    if (id2 < a.n) a.dbg_votes[qi * a.n + id2] = uint8_t((word >> (8 * b)) & 0xffu);
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            const int c = s_cnt;
            publish_items(a, qi, c);
        }
        qi = qn;
    }
}

constexpr int CK_THREADS = 256;
constexpr int CK_WARPS = CK_THREADS / 32;

struct CandKnnArgs {
    const float *X;
    const void *rows;      // rows the distances are computed from (X or its bf16 copy)
    int32_t kfinal;        // neighbours returned (k); a.k holds k + margin when re-ranking
    int32_t rerank;        // re-rank the survivors with float32 rows
    uint32_t row_bytes;    // bytes of one staged row
    int32_t ring;          // rows staged per warp (k_cand_knn)
    uint32_t *status;
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
    const int2 *items;
    const uint32_t *n_items;
    int32_t chunk;
    int32_t max_items_q;   // chunks per query at most (partial-list slots)
    int32_t *done;
    float *part_d;         // partial top-k lists: m x max_items_q x k
    int32_t *part_i;
    const QueryRecord *rec;  // plan mode: Q, outputs and m of the batch
    uint32_t wait_tries;   // tries of each row wait of the distance loop (a test
                           // shortens it so that the wait runs out)
    const int64_t *cand_off;  // optional: query i's list starts at cand + cand_off[i]
};

// First candidate of query qi's list: lists of capq entries one after
// another, or at per-query offsets.
__device__ __forceinline__ const int32_t *cand_list_of(const CandKnnArgs &a, int64_t qi) {
    return a.cand + (a.cand_off != nullptr ? a.cand_off[qi] : qi * int64_t(a.capq));
}

template <int KR>
__global__ void __launch_bounds__(CK_THREADS) k_cand_knn_regs(const CandKnnArgs a0) {
    CandKnnArgs a = a0;
    if (a.rec != nullptr) {
        a.Q = a.rec->Q;
        a.out_ids = a.rec->out_ids;
        a.out_dists = a.rec->out_dists;
        a.m = a.rec->m;
    }
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
        const int c = min(a.ncand[qi], a.capq);
        for (int i = lane; i < a.dpad; i += 32) qv[i] = (i < a.d) ? a.Q[qi * a.d + i] : 0.f;
        __syncwarp();
        WarpTopK<KR> top;
        top.init();
        const int32_t *clist = cand_list_of(a, qi);
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

// One warp per query, candidate rows streamed through a warp-private ring
// of `ring` row slots in shared memory by bulk copies (TMA), each slot with
// its own mbarrier: up to `ring` whole rows are in flight per warp without
// holding them in registers, and warps never wait for one another.
constexpr int CR_WARPS = 4;
constexpr int CR_MAX_RING = 16;

// RK: 0 float32 rows, 1 bfloat16 rows, 2 e4m3 rows with a per-row scale.
// SR > 0 fixes the ring to SR slots at compile time (slot indices and
// parity bits then fold to constants); SR = 0 takes a.ring.
template <int KR, int RK, int SR>
__global__ void __launch_bounds__(CR_WARPS * 32) k_cand_knn(const CandKnnArgs a0) {
    CandKnnArgs a = a0;
    if (a.rec != nullptr) {
        a.Q = a.rec->Q;
        a.out_ids = a.rec->out_ids;
        a.out_dists = a.rec->out_dists;
        a.m = a.rec->m;
    }
    extern __shared__ __align__(16) unsigned char csm[];
    __shared__ __align__(8) uint64_t s_bar[CR_WARPS][CR_MAX_RING];
    __shared__ int32_t s_cid[CR_WARPS][64];  // candidate ids [cbase, cbase + 64) of the item
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int S = SR > 0 ? SR : a.ring;
    const uint32_t row_bytes = a.row_bytes;
    unsigned char *wbase = csm + size_t(warp) * (size_t(a.dpad) * 4 + size_t(S) * row_bytes);
    float *qv = reinterpret_cast<float *>(wbase);
    unsigned char *ring = wbase + size_t(a.dpad) * 4;
    uint64_t *bar = s_bar[warp];
    const float4 *q4 = reinterpret_cast<const float4 *>(qv);
    const unsigned char *Xb = reinterpret_cast<const unsigned char *>(a.rows);
    const int nv4 = a.dpad >> 2;
    const int k = a.k;
    if (lane == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncwarp();
    const uint32_t n_items = *a.n_items;
    const bool qvec = (a.d & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Q) & 15) == 0;
    uint32_t parity = 0;     // bit i: phase parity of slot i
    uint32_t inflight = 0;   // bit i: slot i has a copy outstanding
    bool failed = false;
    int64_t staged_q = -1;
    // the next work item is claimed (and its record read) one item ahead
    uint32_t w = 0;
    if (lane == 0) w = atomicAdd(a.work, 1u);
    w = __shfl_sync(0xffffffffu, w, 0);
    int2 item = make_int2(0, 0);
    int call = 0;
    if (w < n_items) {
        item = a.items[w];
        call = min(a.ncand[item.x], a.capq);
    }
    for (;;) {
        if (w >= n_items) break;
        const int64_t qi = item.x;
        const int ch = item.y;
        uint32_t w_next = 0;
        if (lane == 0) w_next = atomicAdd(a.work, 1u);
        const int csz = item_size(call, a.chunk);
        const int nch = item_count(call, csz);
        const int lo = ch * csz;
        const int c = min(call, lo + csz) - lo;  // candidates of this item
        if (qi != staged_q) {
            __syncwarp();
            if (qvec) {
                const float4 *src = reinterpret_cast<const float4 *>(a.Q + qi * a.d);
                float4 *dst = reinterpret_cast<float4 *>(qv);
                for (int i = lane; i < (a.dpad >> 2); i += 32)
                    dst[i] = 4 * i < a.d ? __ldg(src + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                for (int i = lane; i < a.dpad; i += 32) qv[i] = (i < a.d) ? a.Q[qi * a.d + i] : 0.f;
            }
            staged_q = qi;
        }
        const int32_t *clist = cand_list_of(a, qi) + lo;
        // candidate ids f in [cbase, cbase + 64) in the warp's shared list
        // (f stays below j + 1 + S < cbase + 32 + 17)
        int32_t *cid = s_cid[warp];
        int cbase = 0;
        __syncwarp();
        cid[lane] = lane < c ? __ldg(clist + lane) : 0;
        cid[32 + lane] = 32 + lane < c ? __ldg(clist + 32 + lane) : 0;
        __syncwarp();
        // lane 0 starts the copy of candidate f's row into `slot`
        auto copy_row = [&](int f, int slot) {
            const int32_t id = cid[f - cbase];
            mbar_arrive_expect_tx(&bar[slot], row_bytes);
            bulk_copy_g2s(ring + size_t(slot) * row_bytes, Xb + size_t(id) * row_bytes, row_bytes, &bar[slot]);
        };
        const int prime = c < S ? c : S;
        if (lane == 0)
            for (int f = 0; f < prime; ++f) copy_row(f, f);
        inflight |= (1u << prime) - 1u;
        __syncwarp();
        WarpTopK<KR> top;
        top.init();
        int slot = 0;
        for (int j = 0; j < c; j += 2) {
            if (j - cbase >= 32) {
                const int32_t hi = cid[32 + lane];
                const int32_t nx = cbase + 64 + lane < c ? __ldg(clist + cbase + 64 + lane) : 0;
                __syncwarp();
                cid[lane] = hi;
                cid[32 + lane] = nx;
                cbase += 32;
                __syncwarp();
            }
            const bool two = j + 1 < c;
            const int slot1 = (slot + 1 == S) ? 0 : slot + 1;
            const int32_t id0 = cid[j - cbase];
            const int32_t id1 = two ? cid[j + 1 - cbase] : id0;
            // warp-uniform outcome of the bounded waits
            bool ok = mbar_wait(&bar[slot], (parity >> slot) & 1u, a.wait_tries);
            if (two) ok = mbar_wait(&bar[slot1], (parity >> slot1) & 1u, a.wait_tries) && ok;
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            parity ^= 1u << slot;
            inflight &= ~(1u << slot);
            if (two) {
                parity ^= 1u << slot1;
                inflight &= ~(1u << slot1);
            }
            float dd0, dd1;
            if (RK == 2) {
                const unsigned char *p0 = ring + size_t(slot) * row_bytes;
                const unsigned char *p1 = ring + size_t(two ? slot1 : slot) * row_bytes;
                const float s0 = *reinterpret_cast<const float *>(p0 + row_bytes - 16);
                const float s1 = *reinterpret_cast<const float *>(p1 + row_bytes - 16);
                smem_rows2_sq_dist_fp8(reinterpret_cast<const uint32_t *>(p0),
                                       reinterpret_cast<const uint32_t *>(p1), s0, s1, q4, nv4, lane,
                                       dd0, dd1);
            } else if (RK == 1)
                smem_rows2_sq_dist<uint2>(reinterpret_cast<const uint2 *>(ring + size_t(slot) * row_bytes),
                                          reinterpret_cast<const uint2 *>(ring + size_t(two ? slot1 : slot) * row_bytes),
                                          q4, nv4, lane, dd0, dd1);
            else
                smem_rows2_sq_dist<float4>(reinterpret_cast<const float4 *>(ring + size_t(slot) * row_bytes),
                                           reinterpret_cast<const float4 *>(ring + size_t(two ? slot1 : slot) * row_bytes),
                                           q4, nv4, lane, dd0, dd1);
            __syncwarp();  // every lane has read both slots
            {
                const bool n0 = j + S < c, n1 = two && j + 1 + S < c;
                if (lane == 0) {
                    if (n0) copy_row(j + S, slot);
                    if (n1) copy_row(j + 1 + S, slot1);
                }
                inflight |= (n0 ? 1u << slot : 0u) | (n1 ? 1u << slot1 : 0u);
            }
            top.insert(dd0, id0, k, lane);
            if (two) top.insert(dd1, id1, k, lane);
            slot = two ? ((slot1 + 1 == S) ? 0 : slot1 + 1) : slot1;
        }
        if (failed) break;
        bool finish = nch == 1;
        if (!finish) {
            // publish this chunk's list; the item that completes the query
            // merges every chunk's list into its own
            const int64_t pbase = (qi * a.max_items_q + ch) * int64_t(k);
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int e = r * 32 + lane;
                if (e < k) {
                    a.part_d[pbase + e] = top.d[r];
                    a.part_i[pbase + e] = top.i[r];
                }
            }
            __threadfence();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(a.done + qi, 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            finish = old == nch - 1;
            if (finish) {
                __threadfence();
                for (int ch2 = 0; ch2 < nch; ++ch2) {
                    if (ch2 == ch) continue;
                    const int64_t b2 = (qi * a.max_items_q + ch2) * int64_t(k);
                    for (int e0 = 0; e0 < k; e0 += 32) {
                        float pd = INFINITY;
                        int32_t pi = SENTINEL_ID;
                        if (e0 + lane < k) {
                            pd = __ldcg(a.part_d + b2 + e0 + lane);
                            pi = __ldcg(a.part_i + b2 + e0 + lane);
                        }
                        const int cnt = min(32, k - e0);
                        for (int u = 0; u < cnt; ++u) {
                            const float ud = __shfl_sync(0xffffffffu, pd, u);
                            const int32_t ui = __shfl_sync(0xffffffffu, pi, u);
                            top.insert(ud, ui, k, lane);
                        }
                    }
                }
            }
        }
        if (finish && RK != 0 && a.rerank) {
            // re-rank: exact float32 distances of the k + margin survivors,
            // whose float32 rows stream through the ring, SP reduced-precision
            // slots per float32 row; keep the k smallest
            const uint32_t frow = uint32_t(a.dpad) * 4u;
            const int SP = int((frow + row_bytes - 1) / row_bytes);
            const int S2 = S / SP;
            const unsigned char *Xf = reinterpret_cast<const unsigned char *>(a.X);
            auto sid = [&](int f) -> int32_t {
                int32_t v = SENTINEL_ID;
#pragma unroll
                for (int rr = 0; rr < KR; ++rr) {
                    const int32_t t2 = __shfl_sync(0xffffffffu, top.i[rr], f & 31);
                    if (rr == (f >> 5)) v = t2;
                }
                return v;
            };
            int nsurv = 0;
#pragma unroll
            for (int rr = 0; rr < KR; ++rr)
                nsurv += __popc(__ballot_sync(0xffffffffu, rr * 32 + lane < k && top.i[rr] != SENTINEL_ID));
            auto issue2 = [&](int f, int ss) {
                const int32_t id2 = sid(f);
                if (lane == 0) {
                    mbar_arrive_expect_tx(&bar[SP * ss], frow);
                    bulk_copy_g2s(ring + size_t(SP * ss) * row_bytes, Xf + size_t(id2) * frow, frow,
                                  &bar[SP * ss]);
                }
                inflight |= 1u << (SP * ss);
            };
            const int prime2 = nsurv < S2 ? nsurv : S2;
            for (int f = 0; f < prime2; ++f) issue2(f, f);
            __syncwarp();
            WarpTopK<KR> fin;
            fin.init();
            int ss = 0;
            for (int f = 0; f < nsurv; ++f) {
                const int32_t id2 = sid(f);
                const int bslot = SP * ss;
                if (!__all_sync(0xffffffffu, mbar_wait(&bar[bslot], (parity >> bslot) & 1u))) {
                    failed = true;
                    break;
                }
                parity ^= 1u << bslot;
                inflight &= ~(1u << bslot);
                const float ed = smem_row_sq_dist(
                    reinterpret_cast<const float4 *>(ring + size_t(bslot) * row_bytes), q4, nv4, lane);
                __syncwarp();
                if (f + S2 < nsurv) issue2(f + S2, ss);
                fin.insert(ed, id2, a.kfinal, lane);
                ss = (ss + 1 == S2) ? 0 : ss + 1;
            }
            if (failed) break;
            top = fin;
        }
        if (finish) {
            const int kf = a.kfinal;
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int e = r * 32 + lane;
                if (e < kf) {
                    const bool real = top.i[r] != SENTINEL_ID;
                    a.out_ids[qi * kf + e] = real ? top.i[r] : -1;
                    a.out_dists[qi * kf + e] = real ? sqrtf(top.d[r]) : INFINITY;
                }
            }
        }
        __syncwarp();
        w = __shfl_sync(0xffffffffu, w_next, 0);
        if (w < n_items) {
            item = a.items[w];
            call = min(a.ncand[item.x], a.capq);
        }
    }
    if (failed && lane == 0) {
        atomicOr(a.status, STATUS_TIMEOUT);
        // let copies still in flight land before the warp exits (bounded)
        for (int i = 0; i < S; ++i)
            if ((inflight >> i) & 1u) mbar_wait(&bar[i], (parity >> i) & 1u);
    }
}

// --------------------------------------- candidate search, rows in registers

// acc + (x - q)^2 for the 8 bfloat16 values of one 16-byte chunk x against 8
// float32 query values, two components per packed fma.  Each difference is
// one mixed-precision subtraction (sub.rn.f32.bf16: the bfloat16 operand is
// widened exactly, then one rounding), so (x - q)^2 equals the square of the
// float32 difference q - x of the staged-row kernels.
__device__ __forceinline__ float2 bf16x8_sq_acc(uint4 x, const float (&q)[8], float2 acc) {
    float t0, t1, t2, t3, t4, t5, t6, t7;
    asm("{\n\t"
        ".reg .b16 h<8>;\n\t"
        "mov.b32 {h0, h1}, %8;\n\t"
        "mov.b32 {h2, h3}, %9;\n\t"
        "mov.b32 {h4, h5}, %10;\n\t"
        "mov.b32 {h6, h7}, %11;\n\t"
        "sub.rn.f32.bf16 %0, h0, %12;\n\t"
        "sub.rn.f32.bf16 %1, h1, %13;\n\t"
        "sub.rn.f32.bf16 %2, h2, %14;\n\t"
        "sub.rn.f32.bf16 %3, h3, %15;\n\t"
        "sub.rn.f32.bf16 %4, h4, %16;\n\t"
        "sub.rn.f32.bf16 %5, h5, %17;\n\t"
        "sub.rn.f32.bf16 %6, h6, %18;\n\t"
        "sub.rn.f32.bf16 %7, h7, %19;\n\t"
        "}"
        : "=f"(t0), "=f"(t1), "=f"(t2), "=f"(t3), "=f"(t4), "=f"(t5), "=f"(t6), "=f"(t7)
        : "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w), "f"(q[0]), "f"(q[1]), "f"(q[2]), "f"(q[3]), "f"(q[4]),
          "f"(q[5]), "f"(q[6]), "f"(q[7]));
    acc = __ffma2_rn(make_float2(t0, t1), make_float2(t0, t1), acc);
    acc = __ffma2_rn(make_float2(t2, t3), make_float2(t2, t3), acc);
    acc = __ffma2_rn(make_float2(t4, t5), make_float2(t4, t5), acc);
    acc = __ffma2_rn(make_float2(t6, t7), make_float2(t6, t7), acc);
    return acc;
}

// Sums of two per-lane values over the warp, returned in every lane: lanes
// 0-15 reduce the first and lanes 16-31 the second after one exchange
// (5 shuffles for both instead of 10).
__device__ __forceinline__ void warp_sum2(float s0, float s1, int lane, float &d0, float &d1) {
    const bool hi = (lane & 16) != 0;
    float mine = hi ? s1 : s0;
    const float other = hi ? s0 : s1;
    mine += __shfl_xor_sync(0xffffffffu, other, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    d0 = __shfl_sync(0xffffffffu, mine, 0);
    d1 = __shfl_sync(0xffffffffu, mine, 16);
}

// The same for the 4 float32 values of one 16-byte chunk of a float32 row.
__device__ __forceinline__ float2 f32x4_sq_acc(uint4 x, const float *q, float2 acc) {
    acc = sq_acc2(make_float2(q[0], q[1]), make_float2(__uint_as_float(x.x), __uint_as_float(x.y)), acc);
    return sq_acc2(make_float2(q[2], q[3]), make_float2(__uint_as_float(x.z), __uint_as_float(x.w)), acc);
}
__device__ __forceinline__ float2 chunk_sq_acc(uint4 x, const float (&q)[8], float2 acc) {
    return bf16x8_sq_acc(x, q, acc);
}
__device__ __forceinline__ float2 chunk_sq_acc(uint4 x, const float (&q)[4], float2 acc) {
    return f32x4_sq_acc(x, q, acc);
}

// acc + (q - s x)^2 for the 16 e4m3 values of one 16-byte chunk x of a row
// with scale s (ns = (-s, -s)) against 16 float32 query values: the values
// are widened exactly, then t = q - s x is one fma (the product of a 4-bit
// and a 24-bit significand needs no rounding), then acc += t t.
__device__ __forceinline__ float2 e4m3x16_sq_acc(uint4 x, float2 ns, const float (&q)[16], float2 acc) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 v = e4m3x4_to_float4(w[j]);
        float2 t = __ffma2_rn(ns, make_float2(v.x, v.y), make_float2(q[4 * j], q[4 * j + 1]));
        acc = __ffma2_rn(t, t, acc);
        t = __ffma2_rn(ns, make_float2(v.z, v.w), make_float2(q[4 * j + 2], q[4 * j + 3]));
        acc = __ffma2_rn(t, t, acc);
    }
    return acc;
}

// k_cand_knn for float32 rows (RT = 0), bfloat16 rows (RT = 1) or e4m3 rows
// with a per-row scale (RT = 2) whose
// 16-byte chunks of values (4, 8 or 16 values) number between 32 (U - 1) + 1
// and 32 U (or fewer than 32 with U = 1: lanes past the row idle):
// one warp per (query, chunk of the list) work item, as in k_cand_knn, with
// the rows in a per-warp ring of CB_SLOTS row pairs in shared memory.
// - Lane l owns chunks l, l + 32, ... of every row. It copies its own chunks
//   of each row into the ring with cp.async and later reads back only what it
//   copied. A per-thread wait_group is therefore all the synchronisation: no
//   mbarrier, and no single lane issuing copies for the warp.
// - The query's chunks stay in registers for the whole item.
// - Pairs are copied CB_SLOTS - 1 ahead. Each pair's two sums are reduced
//   together and go into the warp's sorted top-k.
// - An e4m3 row's scale (the float32 after its values) is read by every lane
//   with one broadcast load when the row's pair is copied, so it has arrived
//   when the pair is summed.
// - With a lossy copy (bfloat16 that does not hold X exactly, or e4m3) the
//   item that completes a query re-ranks the k + margin survivors with
//   float32 rows. Each survivor's row goes through the same ring, two rows in
//   flight. Lane l copies the F = 2 or 4 float32 chunks that cover its
//   chunk's 8 or 16 values, so the query registers serve as they are.
constexpr int CB_WARPS = 4;
constexpr int CB_SLOTS = 2;

// 16-byte ring chunks per warp of k_cand_knn_rows for rows of `nchunk` value
// chunks of `vpc` values, `rows` rows per step: CB_SLOTS steps, and with a
// re-rank room for two float32 rows (vpc / 4 float32 chunks per value chunk).
__host__ __device__ constexpr int cb_ring_chunks(int nchunk, int vpc, bool rerank, int rows) {
    return (rerank && 2 * (vpc / 4) > CB_SLOTS * rows ? 2 * (vpc / 4) : CB_SLOTS * rows) * nchunk;
}

// Blocks per SM that k_cand_knn_rows is compiled for (its register cap):
// 7 for k <= 64, which keeps the loop's latency hidden by more resident warps
// (measured against the compiler's default); larger k keeps the default.
__host__ __device__ constexpr int cb_min_blocks(int kr) { return kr <= 2 ? 7 : 1; }

template <int KR, int U, int RT, bool RR, int G>
__global__ void __launch_bounds__(CB_WARPS * 32, cb_min_blocks(KR)) k_cand_knn_rows(const CandKnnArgs a0) {
    constexpr int VPC = RT == 2 ? 16 : RT == 1 ? 8 : 4;  // values per 16-byte chunk
    constexpr int F = VPC / 4;  // float32 chunks per chunk (re-rank)
    constexpr int R = 32 / G;   // rows per slab (one per group of G lanes)
    constexpr int RP = 2 * R;   // rows per step (two slabs)
    static_assert(!RR || RT != 0, "float32 rows need no re-rank");
    static_assert((G == 32 || (U == 1 && (G == 16 || G == 8))), "groups of 8 or 16 lanes take rows of one round");
    CandKnnArgs a = a0;
    if (a.rec != nullptr) {
        a.Q = a.rec->Q;
        a.out_ids = a.rec->out_ids;
        a.out_dists = a.rec->out_dists;
        a.m = a.rec->m;
    }
    extern __shared__ __align__(16) unsigned char cbsm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // 16-byte chunks of values per row; an e4m3 row stores one more (its scale)
    const int nchunk = RT == 2 ? int(a.row_bytes / 16u) - 1 : a.dpad / VPC;
    const int rstride = RT == 2 ? nchunk + 1 : nchunk;
    const uint4 *Xb = reinterpret_cast<const uint4 *>(a.rows);
    uint4 *wring = reinterpret_cast<uint4 *>(cbsm) + size_t(warp) * cb_ring_chunks(nchunk, VPC, RR, RP);
    const int cl = G == 32 ? lane : (lane & (G - 1));  // this lane's chunk of its rows
    const int grp = G == 32 ? 0 : lane / G;            // this lane's row of a slab
    const uint32_t wring_s = smem_u32(wring);
    const int k = a.k;  // survivors kept (k + margin when re-ranking)
    const uint32_t n_items = *a.n_items;
    const bool qvec = (a.d % VPC) == 0 && (reinterpret_cast<uintptr_t>(a.Q) & 15) == 0;
    float qv[U][VPC];
    int64_t staged_q = -1;
    uint32_t w = 0;
    if (lane == 0) w = atomicAdd(a.work, 1u);
    w = __shfl_sync(0xffffffffu, w, 0);
    int2 item = make_int2(0, 0);
    int call = 0;
    if (w < n_items) {
        item = a.items[w];
        call = min(a.ncand[item.x], a.capq);
    }
    while (w < n_items) {
        const int64_t qi = item.x;
        const int ch = item.y;
        uint32_t w_next = 0;
        if (lane == 0) w_next = atomicAdd(a.work, 1u);
        const int csz = item_size(call, a.chunk);
        const int nch = item_count(call, csz);
        const int lo = ch * csz;
        const int c = min(call, lo + csz) - lo;  // candidates of this item
        if (qi != staged_q) {
            const float *qrow = a.Q + qi * a.d;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int cc = cl + 32 * u;
                if (qvec && cc < nchunk && cc * VPC < a.d) {
#pragma unroll
                    for (int h = 0; h < VPC / 4; ++h) {
                        const float4 x = __ldg(reinterpret_cast<const float4 *>(qrow + cc * VPC + 4 * h));
                        qv[u][4 * h] = x.x;
                        qv[u][4 * h + 1] = x.y;
                        qv[u][4 * h + 2] = x.z;
                        qv[u][4 * h + 3] = x.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VPC; ++e) {
                        const int dim = cc * VPC + e;
                        qv[u][e] = (cc < nchunk && dim < a.d) ? __ldg(qrow + dim) : 0.f;
                    }
                }
            }
            staged_q = qi;
        }
        const int32_t *clist = cand_list_of(a, qi) + lo;
        // ids of rows [32 blk, 32 blk + 32) of the item, one per lane
        int blk = 0;
        int32_t ids = lane < c ? __ldg(clist + lane) : 0;
        auto load_blk = [&](int r) {  // r warp-uniform
            if ((r >> 5) != blk) {
                blk = r >> 5;
                const int rr = 32 * blk + lane;
                ids = rr < c ? __ldg(clist + rr) : 0;
            }
        };
        // step p covers rows RP p .. RP p + RP - 1: slab s (0, 1) of it is
        // rows RP p + s R + g, row g of the slab on lane group g.  Each lane
        // copies its chunks of its two rows into slot p % CB_SLOTS (one
        // commit group per step, empty past the item's last step) and loads
        // an e4m3 row's scale.  A row past the item repeats the step's first
        // row (copied, never inserted).  Rounds u < U - 1 are always inside
        // the row (32 (U - 1) < nchunk), only the last one needs a bound.
        auto issue_step = [&](int p, int slot, float2 &sc) {
            const int r0 = RP * p;
            if (r0 < c) {
                load_blk(r0);  // RP divides 32: the step's rows share a block
                const int32_t first = __shfl_sync(0xffffffffu, ids, r0 & 31);
                const int ra = r0 + grp, rb = r0 + R + grp;
                int32_t id0 = __shfl_sync(0xffffffffu, ids, ra & 31);
                int32_t id1 = __shfl_sync(0xffffffffu, ids, rb & 31);
                id0 = ra < c ? id0 : first;
                id1 = rb < c ? id1 : first;
                const uint4 *s0 = Xb + int64_t(id0) * rstride + cl;
                const uint4 *s1 = Xb + int64_t(id1) * rstride + cl;
                if (RT == 2) {
                    sc.x = __ldg(reinterpret_cast<const float *>(Xb + int64_t(id0) * rstride + nchunk));
                    sc.y = __ldg(reinterpret_cast<const float *>(Xb + int64_t(id1) * rstride + nchunk));
                }
                const uint32_t d0 = wring_s + uint32_t((slot * RP + grp) * nchunk + cl) * 16u;
                const uint32_t d1 = d0 + uint32_t(R * nchunk) * 16u;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u < U - 1 || cl + 32 * u < nchunk) {
                        cp_async16_zfill(d0 + uint32_t(32 * u) * 16u, s0 + 32 * u, 16u);
                        cp_async16_zfill(d1 + uint32_t(32 * u) * 16u, s1 + 32 * u, 16u);
                    }
                }
            }
            cp_async_commit();
        };
        WarpTopK<KR> top;
        top.init();
        const int nsteps = (c + RP - 1) / RP;
        int s_issue = 0, s_use = 0;  // slots of the next step to copy and to use
        // scales of the steps in flight (e4m3): scs[j] for step p + j
        float2 scs[CB_SLOTS];
#pragma unroll
        for (int j = 0; j < CB_SLOTS; ++j) scs[j] = make_float2(1.f, 1.f);
#pragma unroll
        for (int p = 0; p < CB_SLOTS - 1; ++p) {
            issue_step(p, s_issue, scs[p]);
            s_issue = s_issue + 1 == CB_SLOTS ? 0 : s_issue + 1;
        }
        for (int p = 0; p < nsteps; ++p) {
            issue_step(p + CB_SLOTS - 1, s_issue, scs[CB_SLOTS - 1]);
            s_issue = s_issue + 1 == CB_SLOTS ? 0 : s_issue + 1;
            // this thread's copies of step p are in (groups of later steps may not be)
            asm volatile("cp.async.wait_group %0;" ::"n"(CB_SLOTS - 1) : "memory");
            const uint4 *r0 = wring + (s_use * RP + grp) * nchunk + cl;
            const uint4 *r1 = r0 + R * nchunk;
            s_use = s_use + 1 == CB_SLOTS ? 0 : s_use + 1;
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
            const float2 ns0 = make_float2(-scs[0].x, -scs[0].x), ns1 = make_float2(-scs[0].y, -scs[0].y);
#pragma unroll
            for (int j = 0; j + 1 < CB_SLOTS; ++j) scs[j] = scs[j + 1];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = u < U - 1 || cl + 32 * u < nchunk;
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                const uint4 x0 = in ? r0[32 * u] : z;
                const uint4 x1 = in ? r1[32 * u] : z;
                if constexpr (RT == 2) {
                    a0 = e4m3x16_sq_acc(x0, ns0, qv[u], a0);
                    a1 = e4m3x16_sq_acc(x1, ns1, qv[u], a1);
                } else {
                    a0 = chunk_sq_acc(x0, qv[u], a0);
                    a1 = chunk_sq_acc(x1, qv[u], a1);
                }
            }
            // both slabs' sums over each group of G lanes: after one exchange
            // the lower half of a group reduces slab 0, the upper half slab 1
            // (with G = 32 the order of warp_sum2)
            const bool hi = (lane & (G / 2)) != 0;
            float part = hi ? a1.x + a1.y : a0.x + a0.y;
            part += __shfl_xor_sync(0xffffffffu, hi ? a0.x + a0.y : a1.x + a1.y, G / 2);
#pragma unroll
            for (int o = G / 4; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            // row RP p + r is row g = r % R of slab s = r / R: its sum is on
            // lane g G + s G / 2 (the ids of a later step may have replaced
            // this step's block)
            load_blk(RP * p);
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const float dr = __shfl_sync(0xffffffffu, part, (r % R) * G + (r / R) * (G / 2));
                const int row = RP * p + r;
                if (row < c) top.insert(dr, __shfl_sync(0xffffffffu, ids, row & 31), k, lane);
            }
        }
        cp_async_wait_all();  // no copy of this item outlives it
        bool finish = nch == 1;
        if (!finish) {
            // publish this chunk's list; the item that completes the query
            // merges every chunk's list into its own
            const int64_t pbase = (qi * a.max_items_q + ch) * int64_t(k);
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int e = r * 32 + lane;
                if (e < k) {
                    a.part_d[pbase + e] = top.d[r];
                    a.part_i[pbase + e] = top.i[r];
                }
            }
            __threadfence();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(a.done + qi, 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            finish = old == nch - 1;
            if (finish) {
                __threadfence();
                for (int ch2 = 0; ch2 < nch; ++ch2) {
                    if (ch2 == ch) continue;
                    const int64_t b2 = (qi * a.max_items_q + ch2) * int64_t(k);
                    for (int e0 = 0; e0 < k; e0 += 32) {
                        float pd = INFINITY;
                        int32_t pi = SENTINEL_ID;
                        if (e0 + lane < k) {
                            pd = __ldcg(a.part_d + b2 + e0 + lane);
                            pi = __ldcg(a.part_i + b2 + e0 + lane);
                        }
                        const int cnt = min(32, k - e0);
                        for (int u = 0; u < cnt; ++u) {
                            const float ud = __shfl_sync(0xffffffffu, pd, u);
                            const int32_t ui = __shfl_sync(0xffffffffu, pi, u);
                            top.insert(ud, ui, k, lane);
                        }
                    }
                }
            }
        }
        if (RR && finish) {
            // re-rank: exact float32 distances of the k + margin survivors,
            // two float32 rows in the ring, the next row copied while this
            // one is summed; keep the kfinal smallest
            const uint4 *Xf = reinterpret_cast<const uint4 *>(a.X);
            const int fstride = a.dpad / 4;  // float32 chunks per row of X
            const int fslot = F * nchunk;    // ring chunks per float32 row
            auto sid = [&](int f) -> int32_t {
                int32_t v = SENTINEL_ID;
#pragma unroll
                for (int rr = 0; rr < KR; ++rr) {
                    const int32_t t2 = __shfl_sync(0xffffffffu, top.i[rr], f & 31);
                    if (rr == (f >> 5)) v = t2;
                }
                return v;
            };
            int nsurv = 0;
#pragma unroll
            for (int rr = 0; rr < KR; ++rr)
                nsurv += __popc(__ballot_sync(0xffffffffu, rr * 32 + lane < k && top.i[rr] != SENTINEL_ID));
            // lane l's float32 chunks F (l + 32 u) + h; those past the row of
            // X (an e4m3 row's last chunk can reach beyond dpad) read as zero.
            // In the ring, chunk h of round u sits at 32 F u + h w_u + l, w_u
            // the lanes of round u (32, or wl in the last): for each (u, h)
            // the lanes touch consecutive 16-byte slots, so neither the
            // copies nor the reads meet bank conflicts.
            const int wl = nchunk - 32 * (U - 1);
            auto slot_of = [&](int u, int h) -> int { return 32 * F * u + h * (u < U - 1 ? 32 : wl) + lane; };
            auto issue_row = [&](int f) {
                if (f < nsurv) {
                    const uint4 *src = Xf + int64_t(sid(f)) * fstride;
                    const uint32_t dst = wring_s + uint32_t((f & 1) * fslot) * 16u;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (u < U - 1 || lane + 32 * u < nchunk) {
#pragma unroll
                            for (int h = 0; h < F; ++h) {
                                const int fc = F * (lane + 32 * u) + h;
                                const bool inrow = RT != 2 || fc < fstride;
                                cp_async16_zfill(dst + uint32_t(slot_of(u, h)) * 16u, inrow ? src + fc : src,
                                                 inrow ? 16u : 0u);
                            }
                        }
                    }
                }
                cp_async_commit();
            };
            WarpTopK<KR> fin;
            fin.init();
            issue_row(0);
            for (int f = 0; f < nsurv; ++f) {
                issue_row(f + 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
                const uint4 *row = wring + (f & 1) * fslot;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u < U - 1 || lane + 32 * u < nchunk) {
#pragma unroll
                        for (int h = 0; h < F; ++h) acc = f32x4_sq_acc(row[slot_of(u, h)], qv[u] + 4 * h, acc);
                    }
                }
                float e0, e1;
                warp_sum2(acc.x + acc.y, 0.f, lane, e0, e1);
                fin.insert(e0, sid(f), a.kfinal, lane);
            }
            cp_async_wait_all();
            top = fin;
        }
        if (finish) {
            const int kf = a.kfinal;
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int e = r * 32 + lane;
                if (e < kf) {
                    const bool real = top.i[r] != SENTINEL_ID;
                    a.out_ids[qi * kf + e] = real ? top.i[r] : -1;
                    a.out_dists[qi * kf + e] = real ? sqrtf(top.d[r]) : INFINITY;
                }
            }
        }
        __syncwarp();
        w = __shfl_sync(0xffffffffu, w_next, 0);
        if (w < n_items) {
            item = a.items[w];
            call = min(a.ncand[item.x], a.capq);
        }
    }
}

// -------------------------------------------------------------- launch ----

namespace {

// Blocks per SM of `func` at `threads` threads and `smem` bytes of dynamic
// shared memory, and the SM count, raising the kernel's shared-memory limit
// first when needed.  The driver queries behind this cost microseconds each,
// which adds up for small batches, so results are kept per (device, kernel,
// threads, bytes).
cudaError_t launch_shape(const void *func, int threads, size_t smem, int device, int *per_sm, int *sms) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> occ;
    static std::map<std::pair<int, const void *>, size_t> limit;
    static std::map<int, int> sm_count;
    std::lock_guard<std::mutex> guard(mu);
    cudaError_t e;
    auto sc = sm_count.find(device);
    if (sc == sm_count.end()) {
        int c = 0;
        if ((e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
        sc = sm_count.emplace(device, c).first;
    }
    *sms = sc->second;
    const auto key = std::make_tuple(device, func, threads, smem);
    const auto hit = occ.find(key);
    if (hit != occ.end()) {
        *per_sm = hit->second;
        return cudaSuccess;
    }
    const auto lk = std::make_pair(device, func);
    const auto li = limit.find(lk);
    if (li == limit.end() || li->second < smem) {
        if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
            return e;
        limit[lk] = smem;
    }
    int p = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, func, threads, smem)) != cudaSuccess) return e;
    occ[key] = p;
    *per_sm = p;
    return cudaSuccess;
}

template <int QB>
cudaError_t launch_route(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const size_t smem = size_t(QB) * size_t(idx->d | 1) * sizeof(float);
    int per_sm = 0, sms = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void *>(k_query_route<QB>), 512, smem, idx->device,
                                 &per_sm, &sms);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (ql.m + QB - 1) / QB;
    const int64_t groups = (ql.n_trees + route_tpi<QB>() - 1) / route_tpi<QB>();
    const int64_t items = tiles * groups;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(items, int64_t(sms) * std::max(per_sm, 1)));
    k_query_route<QB><<<unsigned(blocks), 512, smem, s>>>(ql.Q, ql.m, idx->d, ql.n_trees, idx->l,
                                                         idx->L, idx->rcol, idx->dv,
                                                         idx->split, ql.leaf, ql.proj, idx->status,
                                                         items, ql.rec);
    return cudaGetLastError();
}

// k_route_pairs with NW warps per block and CH pairs per ring slot.
template <int NW, int CH>
cudaError_t launch_route_pairs(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const size_t smem = route_pairs_smem(idx->d, NW, CH);
    int per_sm = 0, sms = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void *>(k_route_pairs<NW, CH>), NW * 32, smem,
                                 idx->device, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    const int64_t units = ((ql.m + RP_QT - 1) / RP_QT) * int64_t(ql.n_trees);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(units, int64_t(sms) * std::max(per_sm, 1)));
    k_route_pairs<NW, CH><<<unsigned(blocks), NW * 32, smem, s>>>(ql.Q, ql.m, idx->d, ql.n_trees, idx->l,
                                                                 idx->L, idx->rcol, idx->dv, idx->split,
                                                                 ql.leaf, ql.proj, idx->status, ql.rec);
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
    // + the sentinel's word (and 3 unused) and a spare word per lane
    size_t region = std::max(size_t(cnt_words + 36) * 4, merge_bytes);
    region = (region + 15) & ~size_t(15);
    smem = region + size_t(idx->dpad) * 4 + size_t(VS_WARPS) * WBUF * 4 + size_t(4 * ql.n_trees) * 4;
    int per_sm = 0, sms = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void *>(k_vote_search<KR>), VS_THREADS, smem,
                                 idx->device, &per_sm, &sms);
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
    a.leaf4 = idx->leaf4;
    a.leaf_off4 = idx->leaf_off4;
    a.s4 = idx->vote_s4;
    a.sentinel = vote_sentinel(idx->n);
    a.chunk_bnd = idx->chunk_bnd;
    a.n_chunks = idx->n_chunks;
    a.L = idx->L;
    a.rec = ql.rec;
    return cudaSuccess;
}

template <int KR>
cudaError_t launch_vote(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    VoteSearchArgs a;
    size_t smem = 0;
    int64_t blocks = 0;
    uint32_t *ctr = ql.counters ? ql.counters : idx->status;
    cudaError_t e = plan_vote<KR>(idx, ql, ctr + 1, a, smem, blocks);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ctr + 1, 0, sizeof(uint32_t), s);
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

// Largest dynamic shared memory of one block on sm_103 (227 KB).
constexpr size_t SMEM_BLOCK_MAX = 232448;

cudaError_t launch_route_any(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    // two queries per lane when a 64-query tile fits (the split descent
    // needs at least one level): 32 warps per block where their rings fit
    // beside the tile (d <= 780), else 16 (d <= 844)
    if (idx->l >= 1) {
        if (route_pairs_smem(idx->d, 32, 64) <= SMEM_BLOCK_MAX) return launch_route_pairs<32, 64>(idx, ql, s);
        if (route_pairs_smem(idx->d, 16, 64) <= SMEM_BLOCK_MAX) return launch_route_pairs<16, 64>(idx, ql, s);
    }
    // else as many queries per block (up to 32, one per lane) as fit in ~110 KB
    const int64_t per_q = int64_t(idx->d) * 4;
    if (per_q * 32 <= 110 * 1024) return launch_route<32>(idx, ql, s);
    if (per_q * 16 <= 110 * 1024) return launch_route<16>(idx, ql, s);
    if (per_q * 8 <= 160 * 1024) return launch_route<8>(idx, ql, s);
    if (per_q * 4 <= 160 * 1024) return launch_route<4>(idx, ql, s);
    if (per_q * 2 <= 200 * 1024) return launch_route<2>(idx, ql, s);
    return launch_route<1>(idx, ql, s);
}

cudaError_t launch_vote_emit(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const int cnt_words = vote_cnt_words(idx->n);
    const bool flat = idx->leaf4 != nullptr;
    // chunked: per-tree windows, or windows over the chunk's segments laid
    // end to end when a leaf's share of a chunk is short (windows would run
    // mostly empty)
    const int64_t leaf_len = (idx->n + idx->L - 1) / idx->L;
    const int64_t chunks = (idx->n + CH_IDS - 1) / CH_IDS;
    const bool packed = !flat && leaf_len < 48 * chunks;
    // one window per leaf and at least 32 16-byte units in every leaf: leaf
    // sizes at depth l are floor(n / 2^l) or one more, and units are
    // ceil(size / 4) (the vote layout pads with the sentinel)
    const int64_t min_units = (idx->n / idx->L + 3) / 4;
    const bool one = flat && (idx->vote_win + 1) / 2 <= 1 && min_units >= 32;
    // hashed counters only on request: the caller (mrpt_query_ex, plan
    // creation) checked that the T leaves of a query hold at most
    // MRPT_VOTE_HASH_ENTRIES entries and that ids + 1 take 24 bits.  The
    // id-chunked counters measured faster where both apply.
    static_assert(MRPT_VOTE_HASH_ENTRIES <= VH_SLOTS * 3 / 4, "the hash table must not fill");
    const bool hashed = ql.vote_table == MRPT_VOTE_HASH;
    if (hashed) {
        VoteEmitArgs h{};
        h.n = idx->n;
        h.leaf_of_q = ql.leaf;
        h.T_use = ql.n_trees;
        h.leaf_off = idx->leaf_off;
        h.leaf_ids = idx->leaf_ids;
        h.m = ql.m;
        h.v = ql.v;
        h.cand = ql.cand_list;
        h.capq = ql.capq;
        h.ncand = ql.ncand;
        uint32_t *hc = ql.counters ? ql.counters : idx->status;
        h.work = hc + 1;
        h.rec = ql.rec;
        h.items = ql.items;
        h.n_items = hc + 5;
        h.chunk = ql.chunk;
        h.done = ql.done;
        h.dbg_votes = ql.votes;
        h.dbg_ncand = ql.n_cand;
        h.dbg_cand = ql.cand;
        h.cand_cap = ql.cand_cap;
        // 128-entry windows of the longest leaf, whose start lies up to 3
        // entries past a 16-byte boundary
        h.win = int((leaf_len + 3 + VE_WIN - 1) / VE_WIN);
        const size_t hsmem = size_t(VH_SLOTS) * 4 + size_t(ql.n_trees) * 16;
        int hper = 0, hsms = 0;
        cudaError_t he = launch_shape(reinterpret_cast<const void *>(k_vote_hash), VH_THREADS, hsmem, idx->device,
                                      &hper, &hsms);
        if (he != cudaSuccess) return he;
        const int64_t hblocks = std::max<int64_t>(1, std::min<int64_t>(ql.m, int64_t(hsms) * std::max(hper, 1)));
        k_vote_hash<<<unsigned(hblocks), VH_THREADS, hsmem, s>>>(h);
        return cudaGetLastError();
    }
    auto kern = flat ? (one ? k_vote_flat<true> : k_vote_flat<false>) : packed ? k_vote_packed : k_vote_emit;
    const size_t smem = flat     ? size_t(cnt_words + 36) * 4 + size_t(ql.n_trees) * 8
                        : packed ? size_t(cnt_words + 32) * 4 + size_t(5 * ql.n_trees + 1) * 4
                                 : size_t(cnt_words + 32) * 4 + size_t(ql.n_trees) * 16 +
                                       size_t(5 * ql.n_trees + 1) * 4;
    int per_sm = 0, sms = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void *>(kern), VE_THREADS, smem, idx->device, &per_sm,
                                 &sms);
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
    uint32_t *ctr = ql.counters ? ql.counters : idx->status;
    a.work = ctr + 1;
    a.rec = ql.rec;
    a.cnt_words = cnt_words;
    a.items = ql.items;
    a.n_items = ctr + 5;
    a.chunk = ql.chunk;
    a.done = ql.done;
    a.dbg_votes = ql.votes;
    a.dbg_ncand = ql.n_cand;
    a.dbg_cand = ql.cand;
    a.cand_cap = ql.cand_cap;
    a.leaf4 = idx->leaf4;
    a.leaf_off4 = idx->leaf_off4;
    a.s4 = idx->vote_s4;
    // 256-entry windows per leaf (vote_win counts 128-entry ones);
    // i / win = (i * win_magic) >> 32 for every window index i < T win
    a.win = std::max((idx->vote_win + 1) / 2, 1);
    a.win_magic = ((uint64_t(1) << 32) + uint64_t(a.win) - 1) / uint64_t(a.win);
    a.sentinel = vote_sentinel(idx->n);
    a.chunk_bnd = idx->chunk_bnd;
    a.n_chunks = idx->n_chunks;
    a.L = idx->L;
    kern<<<unsigned(blocks), VE_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KR, int RK>
cudaError_t launch_cand_knn(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const size_t row_bytes = RK == 2 ? size_t(idx->row8_bytes) : size_t(idx->dpad) * (RK == 1 ? 2 : 4);
    constexpr bool BF16 = RK != 0;  // reduced-precision rows (staged path only)
    // rows staged per warp: two (one pair in flight) by default -- the
    // kernel hides latency with resident warps rather than ring depth, so
    // the smallest ring (most warps per SM) measured fastest
    int ring = ql.ring > 0 ? ql.ring : 2;
    // a re-rank streams float32 rows through the ring: it must hold one
    const bool rerank = RK == 2 || (RK == 1 && !idx->bf16_exact);
    if (rerank) {
        const int sp = int((size_t(idx->dpad) * 4 + row_bytes - 1) / row_bytes);
        ring = std::max(ring, std::min(sp, CR_MAX_RING));
    }
    const size_t per_warp = size_t(idx->dpad) * 4 + size_t(ring) * row_bytes;
    CandKnnArgs a{};
    a.X = idx->X;
    a.rows = RK == 2   ? static_cast<const void *>(idx->X8)
             : RK == 1 ? static_cast<const void *>(idx->Xb)
                       : static_cast<const void *>(idx->X);
    a.row_bytes = uint32_t(row_bytes);
    a.kfinal = ql.k;
    a.dpad = idx->dpad;
    a.Q = ql.Q;
    a.m = ql.m;
    a.d = idx->d;
    a.cand = ql.cand_list;
    a.capq = ql.capq;
    a.ncand = ql.ncand;
    // a lossless bfloat16 copy gives float32 distances up to summation
    // order: no survivors beyond k and no re-rank are needed
    a.rerank = rerank ? 1 : 0;
    a.k = ql.k + (a.rerank ? ql.margin : 0);
    a.out_ids = ql.out_ids;
    a.out_dists = ql.out_dists;
    uint32_t *ctr = ql.counters ? ql.counters : idx->status;
    a.work = ctr + 2;
    a.ring = ring;
    a.status = idx->status;
    a.rec = ql.rec;
    a.items = ql.items;
    a.n_items = ctr + 5;
    a.chunk = ql.chunk;
    a.max_items_q = ql.max_items_q;
    a.done = ql.done;
    a.part_d = ql.part_d;
    a.part_i = ql.part_i;
    a.wait_tries = debug_row_wait_tries();
    a.cand_off = ql.cand_off;
    int sms = 0, per_sm = 0;
    cudaError_t e;
    // rows of at least 8 16-byte chunks of values (float32 dpad >= 32,
    // bfloat16 dpad >= 64, e4m3 dpad > 112) and dpad <= 1024: each lane
    // copies its own chunks (k_cand_knn_rows); rows of at most 16 chunks go
    // to groups of 16 or 8 lanes, two or four rows per slab
    const int vpc = RK == 2 ? 16 : RK == 1 ? 8 : 4;
    const int nchunk = RK == 2 ? int(row_bytes / 16) - 1 : idx->dpad / vpc;
    if (nchunk >= 8 && idx->dpad <= 1024) {
        const int U = (nchunk + 31) / 32;
        const int G = nchunk <= 8 ? 8 : nchunk <= 16 ? 16 : 32;
        const void *kern = nullptr;
#define ROWS_KERN(U_, RT_, RR_, G_) reinterpret_cast<const void *>(k_cand_knn_rows<KR, U_, RT_, RR_, G_>)
        if (RK == 2) {
            kern = G == 8 ? ROWS_KERN(1, 2, true, 8) : G == 16 ? ROWS_KERN(1, 2, true, 16)
                   : U == 1 ? ROWS_KERN(1, 2, true, 32) : ROWS_KERN(2, 2, true, 32);
        } else if (RK == 1 && rerank) {
            kern = G == 8    ? ROWS_KERN(1, 1, true, 8)
                   : G == 16 ? ROWS_KERN(1, 1, true, 16)
                   : U == 1  ? ROWS_KERN(1, 1, true, 32)
                   : U == 2  ? ROWS_KERN(2, 1, true, 32)
                   : U == 3  ? ROWS_KERN(3, 1, true, 32)
                             : ROWS_KERN(4, 1, true, 32);
        } else if (RK == 1) {
            kern = G == 8    ? ROWS_KERN(1, 1, false, 8)
                   : G == 16 ? ROWS_KERN(1, 1, false, 16)
                   : U == 1  ? ROWS_KERN(1, 1, false, 32)
                   : U == 2  ? ROWS_KERN(2, 1, false, 32)
                   : U == 3  ? ROWS_KERN(3, 1, false, 32)
                             : ROWS_KERN(4, 1, false, 32);
        } else {
            const void *by_u[8] = {ROWS_KERN(1, 0, false, 32), ROWS_KERN(2, 0, false, 32),
                                   ROWS_KERN(3, 0, false, 32), ROWS_KERN(4, 0, false, 32),
                                   ROWS_KERN(5, 0, false, 32), ROWS_KERN(6, 0, false, 32),
                                   ROWS_KERN(7, 0, false, 32), ROWS_KERN(8, 0, false, 32)};
            kern = G == 8 ? ROWS_KERN(1, 0, false, 8) : G == 16 ? ROWS_KERN(1, 0, false, 16) : by_u[U - 1];
        }
#undef ROWS_KERN
        const int rows = 2 * (32 / G);
        const size_t smem = size_t(CB_WARPS) * size_t(cb_ring_chunks(nchunk, vpc, rerank, rows)) * 16;
        e = launch_shape(kern, CB_WARPS * 32, smem, idx->device, &per_sm, &sms);
        if (e != cudaSuccess) return e;
        const int64_t blocks = std::max<int64_t>(
            1, std::min<int64_t>((ql.m * 4 + CB_WARPS - 1) / CB_WARPS, int64_t(sms) * std::max(per_sm, 1)));
        void *args[] = {&a};
        return cudaLaunchKernel(kern, dim3(unsigned(blocks)), dim3(CB_WARPS * 32), args, smem, s);
    }
    if (BF16 || CR_WARPS * per_warp <= 200 * 1024) {
        const size_t smem = CR_WARPS * per_warp;
        // the default two-slot ring of k <= 64 as a compile-time constant
        auto kern = (ring == 2 && KR <= 2) ? k_cand_knn<KR, RK, 2> : k_cand_knn<KR, RK, 0>;
        e = launch_shape(reinterpret_cast<const void *>(kern), CR_WARPS * 32, smem, idx->device, &per_sm, &sms);
        if (e != cudaSuccess) return e;
        const int64_t blocks = std::max<int64_t>(
            1, std::min<int64_t>((ql.m + CR_WARPS - 1) / CR_WARPS, int64_t(sms) * std::max(per_sm, 1)));
        kern<<<unsigned(blocks), CR_WARPS * 32, smem, s>>>(a);
        return cudaGetLastError();
    }
    // float32 rows too long to stage: register path
    const size_t smem = size_t(CK_WARPS) * size_t(idx->dpad) * 4;
    e = launch_shape(reinterpret_cast<const void *>(k_cand_knn_regs<KR>), CK_THREADS, smem, idx->device, &per_sm,
                     &sms);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>((ql.m + CK_WARPS - 1) / CK_WARPS, int64_t(sms) * std::max(per_sm, 1)));
    k_cand_knn_regs<KR><<<unsigned(blocks), CK_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// k_cand_knn for ql's precision and k (the candidate lists, |S| and work
// items already written).
cudaError_t launch_search_any(const mrpt_index *idx, const QueryLaunch &ql, cudaStream_t s) {
    const int kr = (ql.k + 31) / 32;
    if (ql.precision == 1) {
        // survivors kept for the re-rank (none beyond k when it is skipped)
        const int krs = (ql.k + (idx->bf16_exact ? 0 : ql.margin) + 31) / 32;
        if (krs <= 1) return launch_cand_knn<1, 1>(idx, ql, s);
        if (krs <= 2) return launch_cand_knn<2, 1>(idx, ql, s);
        if (krs <= 4) return launch_cand_knn<4, 1>(idx, ql, s);
        return launch_cand_knn<8, 1>(idx, ql, s);
    }
    if (ql.precision == 2) {
        const int krs = (ql.k + ql.margin + 31) / 32;
        if (krs <= 1) return launch_cand_knn<1, 2>(idx, ql, s);
        if (krs <= 2) return launch_cand_knn<2, 2>(idx, ql, s);
        if (krs <= 4) return launch_cand_knn<4, 2>(idx, ql, s);
        return launch_cand_knn<8, 2>(idx, ql, s);
    }
    if (kr <= 1) return launch_cand_knn<1, 0>(idx, ql, s);
    if (kr <= 2) return launch_cand_knn<2, 0>(idx, ql, s);
    if (kr <= 4) return launch_cand_knn<4, 0>(idx, ql, s);
    return launch_cand_knn<8, 0>(idx, ql, s);
}

}  // namespace

int launch_search_only(mrpt_index *idx, const QueryLaunch &ql) {
    if (ql.m == 0) return MRPT_OK;
    const cudaError_t e = launch_search_any(idx, ql, ql.use_stream ? ql.stream : idx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "k_cand_knn");
    return MRPT_OK;
}

int launch_route_only(mrpt_index *idx, const QueryLaunch &ql) {
    if (ql.m == 0) return MRPT_OK;
    const cudaError_t e = launch_route_any(idx, ql, ql.use_stream ? ql.stream : idx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "routing kernel");
    return MRPT_OK;
}

int launch_query(mrpt_index *idx, const QueryLaunch &ql) {
    cudaStream_t s = ql.use_stream ? ql.stream : idx->stream;
    if (ql.m == 0) return MRPT_OK;
    cudaError_t e;
    if (ql.stage_ms) {
        for (int i = 0; i < 4; ++i)
            if (!idx->ev[i]) MRPT_CUDA_TRY(cudaEventCreate(&idx->ev[i]));
        MRPT_CUDA_TRY(cudaEventRecord(idx->ev[0], s));
    }
    if (!ql.routed) {
        e = launch_route_any(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "routing kernel");
    }
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
        // work counters [1] vote/emit, [2] candidate search, [3], [4]
        // unused, [5] candidate-search work items
        MRPT_CUDA_TRY(cudaMemsetAsync((ql.counters ? ql.counters : idx->status) + 1, 0,
                                      5 * sizeof(uint32_t), s));
        e = launch_vote_emit(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_vote_emit");
        if (ql.stage_ms) MRPT_CUDA_TRY(cudaEventRecord(idx->ev[2], s));
        e = launch_search_any(idx, ql, s);
        if (e != cudaSuccess) return cuda_fail(e, "k_cand_knn");
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
    cudaError_t e = launch_route_any(idx, ql, s);
    if (e != cudaSuccess) return cuda_fail(e, "routing kernel");
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

namespace mrpt {

int make_bf16_copy(mrpt_index *idx) {
    const int64_t count = idx->n * int64_t(idx->dpad);
    if (!idx->Xb) {
        int rc = dev_alloc(reinterpret_cast<void **>(&idx->Xb), size_t(count) * 2, "bfloat16 copy");
        if (rc) return rc;
        idx->device_bytes += count * 2;
    }
    const int blocks = int(std::min<int64_t>((count + 255) / 256, 152 * 16));
    uint32_t *flag = idx->status + 6;
    MRPT_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(uint32_t), idx->stream));
    k_to_bf16<<<blocks, 256, 0, idx->stream>>>(idx->X, reinterpret_cast<__nv_bfloat16 *>(idx->Xb), count,
                                                flag);
    MRPT_CUDA_TRY(cudaGetLastError());
    uint32_t lossy = 1;
    MRPT_CUDA_TRY(cudaMemcpyAsync(&lossy, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, idx->stream));
    MRPT_CUDA_TRY(cudaStreamSynchronize(idx->stream));
    idx->bf16_exact = lossy == 0;
    return MRPT_OK;
}

}  // namespace mrpt

namespace mrpt {

// Writes a plan's batch record on the stream; the record travels in the
// launch arguments, so the host object may be reused at once.
__global__ void k_set_record(QueryRecord *rec, QueryRecord r) { *rec = r; }

int set_record(QueryRecord *rec, const QueryRecord &r, cudaStream_t s) {
    k_set_record<<<1, 1, 0, s>>>(rec, r);
    MRPT_CUDA_TRY(cudaGetLastError());
    return MRPT_OK;
}

}  // namespace mrpt

namespace mrpt {

int make_fp8_copy(mrpt_index *idx) {
    idx->row8_bytes = ((idx->dpad + 15) & ~15) + 16;
    if (!idx->X8) {
        const size_t bytes = size_t(idx->n) * size_t(idx->row8_bytes);
        int rc = dev_alloc(reinterpret_cast<void **>(&idx->X8), bytes, "e4m3 copy");
        if (rc) return rc;
        idx->device_bytes += int64_t(bytes);
    }
    const int blocks = int(std::min<int64_t>((idx->n * 32 + 255) / 256, 152 * 16));
    k_to_fp8<<<blocks, 256, 0, idx->stream>>>(idx->X, idx->n, idx->dpad, idx->X8, idx->row8_bytes);
    MRPT_CUDA_TRY(cudaGetLastError());
    MRPT_CUDA_TRY(cudaStreamSynchronize(idx->stream));
    return MRPT_OK;
}

}  // namespace mrpt
