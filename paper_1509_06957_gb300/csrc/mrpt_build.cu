// Index construction (Sec. II, Algorithms 1-2) on sm_103a.
//
//   1. generate_random_matrix  (host)  sparse R, one vector per tree level
//                                      (Sec. II-B, II-C)
//   2. k_project_build                 P = XR for all n points and T*l
//                                      vectors (Algorithm 1), column-major
//   3. k_gather_keys + k_split_level   level-synchronous median split of
//      (x l)                           every node of every tree (Algorithm 2,
//                                      order-based median of Sec. II-A)
//   4. k_leaf_offsets                  leaf boundaries (identical per tree)
//
// Each node's members are kept as a contiguous segment of a per-tree
// permutation.  A node is split by a radix select of the rank-ceil(c/2)
// element under the (projection, id) order followed by a stable partition,
// so members stay in ascending id order and leaves need no final sort.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "mrpt_internal.cuh"

namespace mrpt {

// --------------------------------------------------------- random matrix --

namespace {

inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    // output number i (0-based) of SplitMix64 whose state starts at `seed`
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

inline double u53_closed_open(uint64_t x) { return double(x >> 11) * 0x1.0p-53; }
inline double u53_open_closed(uint64_t x) { return (double(x >> 11) + 1.0) * 0x1.0p-53; }

}  // namespace

int32_t fixed_nonzeros(float density, int32_t d) {
    // ceil(a d) in [1, d]; a arrives as a float, so a relative allowance of
    // 1e-6 keeps e.g. float(1/sqrt(784)) * 784 = 28.0000013 at 28
    double k = std::ceil(double(density) * double(d) * (1.0 - 1e-6));
    k = std::min(std::max(k, 1.0), double(d));
    return int32_t(k);
}

void generate_random_matrix(int32_t T, int32_t l, int32_t d, float density, uint64_t seed,
                            int32_t sparsity, int32_t tree_offset, std::vector<int32_t> &col_off,
                            std::vector<int32_t> &dim, std::vector<float> &val) {
    const double a = double(density);
    const double tau = 2.0 * 3.14159265358979323846;
    const int64_t ncols = int64_t(T) * l;
    const bool fixed = sparsity == MRPT_SPARSITY_FIXED;
    const int32_t k = fixed ? fixed_nonzeros(density, d) : 0;
    col_off.assign(size_t(ncols + 1), 0);
    dim.clear();
    val.clear();
    dim.reserve(fixed ? size_t(ncols * k) : size_t(double(ncols) * d * a * 1.2 + 16));
    val.reserve(dim.capacity());
    std::vector<std::pair<double, int32_t>> draws(fixed ? size_t(d) : 0);
    std::vector<int32_t> pick(fixed ? size_t(k) : 0);
    auto normal_at = [&](uint64_t ctr) {
        const double u1 = u53_open_closed(splitmix64_at(seed, ctr + 1));
        const double u2 = u53_closed_open(splitmix64_at(seed, ctr + 2));
        return float(std::sqrt(-2.0 * std::log(u1)) * std::cos(tau * u2));
    };
    for (int64_t c = 0; c < ncols; ++c) {
        col_off[size_t(c)] = int32_t(dim.size());
        // column c of this index is column tree_offset * l + c of the
        // random source (tree t of the index is tree tree_offset + t)
        const uint64_t base = 3ULL * (uint64_t(c) + uint64_t(tree_offset) * uint64_t(l)) * uint64_t(d);
        if (fixed) {
            // the k dimensions with the smallest (first draw, dimension)
            for (int32_t i = 0; i < d; ++i)
                draws[size_t(i)] = {u53_closed_open(splitmix64_at(seed, base + 3ULL * uint64_t(i))), i};
            std::nth_element(draws.begin(), draws.begin() + (k - 1), draws.end());
            for (int32_t r = 0; r < k; ++r) pick[size_t(r)] = draws[size_t(r)].second;
            std::sort(pick.begin(), pick.end());
            for (int32_t i : pick) {
                dim.push_back(i);
                val.push_back(normal_at(base + 3ULL * uint64_t(i)));
            }
            continue;
        }
        for (int32_t i = 0; i < d; ++i) {
            const uint64_t ctr = base + 3ULL * uint64_t(i);
            if (u53_closed_open(splitmix64_at(seed, ctr)) < a) {
                dim.push_back(i);
                val.push_back(normal_at(ctr));
            }
        }
    }
    col_off[size_t(ncols)] = int32_t(dim.size());
}

// ------------------------------------------------------------ finiteness --

__global__ void k_check_finite(const float *__restrict__ X, int64_t rows, int32_t stride,
                               int32_t cols, uint32_t *__restrict__ flag) {
    const int64_t total = rows * int64_t(cols);
    bool bad = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = i / cols;
        const int64_t c = i - r * cols;
        bad |= !isfinite(X[r * stride + c]);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

int check_finite(const float *X, int64_t rows, int32_t stride, int32_t cols, cudaStream_t s,
                 bool *nonfinite) {
    uint32_t *flag = nullptr;
    int rc = dev_alloc((void **)&flag, sizeof(uint32_t), "finiteness flag");
    if (rc) return rc;
    uint32_t h = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess && rows > 0) {
        const int64_t total = rows * int64_t(cols);
        const int blocks = int(std::min<int64_t>((total + 255) / 256, 152 * 16));
        k_check_finite<<<blocks, 256, 0, s>>>(X, rows, stride, cols, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "finiteness check");
    *nonfinite = h != 0;
    return MRPT_OK;
}

// ------------------------------------------------------------ projection --

// P = X R (Algorithm 1) for RB rows per block: the rows are staged in shared
// memory with an odd row stride (conflict-free when 32 lanes read the same
// dimension of different rows); lane (r, g) of a warp computes row r of
// column group g.  Every projection is an fmaf chain over the column's
// nonzeros in ascending dimension from +0.0f.  Output is column-major,
// Pcm[c * n + x], so that a node's keys for one level are one column.
template <int RB>
__global__ void __launch_bounds__(1024) k_project_build(
    const float *__restrict__ X, int64_t n, int32_t dpad, int32_t d,
    const int32_t *__restrict__ col_off, const int32_t *__restrict__ dim,
    const float *__restrict__ val, int32_t ncols, float *__restrict__ Pcm) {
    extern __shared__ float xs[];
    const int stride = d | 1;
    const int64_t row0 = int64_t(blockIdx.x) * RB;
    const int rows = int((n - row0) < RB ? (n - row0) : int64_t(RB));
    const int v4 = dpad >> 2;  // float4 per stored row
    for (int i = threadIdx.x; i < RB * v4; i += blockDim.x) {
        const int r = i / v4;
        const int c4 = i - r * v4;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows) x = reinterpret_cast<const float4 *>(X + (row0 + r) * dpad)[c4];
        const int c = c4 * 4;
        float *dst = xs + r * stride + c;
        if (c + 0 < d) dst[0] = x.x;
        if (c + 1 < d) dst[1] = x.y;
        if (c + 2 < d) dst[2] = x.z;
        if (c + 3 < d) dst[3] = x.w;
    }
    __syncthreads();
    constexpr int G = 32 / RB;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int r = lane % RB;
    const int g = lane / RB;
    const float *xr = xs + r * stride;
    for (int c = warp * G + g; c < ncols; c += nwarps * G) {
        float acc = 0.0f;
        const int e1 = col_off[c + 1];
        for (int e = col_off[c]; e < e1; ++e) acc = __fmaf_rn(xr[dim[e]], val[e], acc);
        if (r < rows) Pcm[int64_t(c) * n + row0 + r] = acc;
    }
}

// ----------------------------------------------------------- median split --

// Order-preserving map of a float to uint32 (-0 is folded into +0 first so
// that equal floats map to equal keys).
__device__ __forceinline__ uint32_t ordered_bits(float f) {
    uint32_t u = (f == 0.0f) ? 0u : __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unordered_float(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Node b at `level`: offset and size of its segment.  Sizes follow the
// ceil-left halving of the order-based median (left gets ceil(c/2)).
__device__ __forceinline__ void node_segment(int64_t n, int level, int64_t b, int64_t &off,
                                             int64_t &c) {
    off = 0;
    c = n;
    for (int s = level - 1; s >= 0; --s) {
        const int64_t h = (c + 1) >> 1;
        if ((b >> s) & 1) {
            off += h;
            c -= h;
        } else {
            c = h;
        }
    }
}

// One block per (tree, node) of `level`.  The node's members in[0..c) are
// in ascending id order.  Find the member of rank ceil(c/2)-1 under the
// composite key (ordered projection << 32 | id) by an 8-bit radix select,
// record its projection as the node's split, and stably partition members
// with composite <= pivot to the left part out[0..ceil(c/2)).
// The level's keys in permutation order: okeys[t n + i] = ordered bits of
// tree t's level projection of point perm[t n + i].  One gather per level,
// after which every pass of the split streams contiguous memory.
__global__ void k_gather_keys(const float *__restrict__ Pcm, int64_t n, int32_t l, int32_t level,
                              int32_t T, const int32_t *__restrict__ perm,
                              uint32_t *__restrict__ okeys) {
    const int64_t total = n * T;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = i / n;
        okeys[i] = ordered_bits(__ldg(Pcm + (t * l + level) * n + perm[i]));
    }
}

// WH (nodes of 16,384 points or more, 1,024-thread blocks): radix digits
// are counted in one histogram per warp, a plain shared atomic per member,
// summed after each pass; otherwise equal digits within a warp are
// aggregated into one atomic on a single histogram.
template <bool WH>
__global__ void __launch_bounds__(1024) k_split_level(
    const float *__restrict__ Pcm, const uint32_t *__restrict__ okeys, int64_t n, int32_t l,
    int32_t level,
    const int32_t *__restrict__ perm_in, int32_t *__restrict__ perm_out,
    float *__restrict__ split, int64_t L) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t whist[WH ? 32 * 256 : 1];  // per-warp digit counts (WH)
    __shared__ uint32_t s_bucket, s_count;
    __shared__ int64_t s_rank;
    __shared__ unsigned long long s_pivot;
    __shared__ uint32_t s_wl[32], s_wr[32];

    const int64_t nodes = int64_t(1) << level;
    const int64_t seg = blockIdx.x;
    const int64_t t = seg / nodes;
    const int64_t b = seg - t * nodes;
    int64_t off, c;
    node_segment(n, level, b, off, c);
    (void)Pcm;
    const uint32_t *okey = okeys + t * n + off;
    const int32_t *in = perm_in + t * n + off;
    int32_t *out = perm_out + t * n + off;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int bd = blockDim.x;
    const int nwarps = bd >> 5;

    auto composite = [&](int64_t i) -> uint64_t {
        return (uint64_t(okey[i]) << 32) | uint32_t(in[i]);
    };

    // ---- radix select of rank r (0-based)
    uint64_t prefix = 0, mask = 0;
    int64_t rank = (c + 1) / 2 - 1;
    bool unique = false;
    constexpr bool per_warp = WH;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        if constexpr (per_warp) {
            for (int i = tid; i < nwarps * 256; i += bd) whist[i] = 0;
        } else {
            for (int i = tid; i < 256; i += bd) hist[i] = 0;
        }
        __syncthreads();
        if constexpr (per_warp) {
            uint32_t *wh = whist + warp * 256;
            for (int64_t base = 0; base < c; base += bd) {
                const int64_t i = base + tid;
                if (i < c) {
                    const uint64_t K = composite(i);
                    if ((K & mask) == prefix) atomicAdd(wh + (uint32_t(K >> shift) & 0xffu), 1u);
                }
            }
            __syncthreads();
            for (int d = tid; d < 256; d += bd) {
                uint32_t sum = 0;
                for (int w = 0; w < nwarps; ++w) sum += whist[w * 256 + d];
                hist[d] = sum;
            }
        } else {
            for (int64_t base = 0; base < c; base += bd) {
                const int64_t i = base + tid;
                const bool in_seg = i < c;
                uint32_t digit = 0;
                bool hit = false;
                if (in_seg) {
                    const uint64_t K = composite(i);
                    hit = (K & mask) == prefix;
                    digit = uint32_t(K >> shift) & 0xffu;
                }
                // warp-aggregated increment: one atomic per distinct digit
                const unsigned act = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const unsigned peers = __match_any_sync(act, digit);
                    if ((peers & ((1u << lane) - 1u)) == 0) atomicAdd(&hist[digit], __popc(peers));
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t sum = 0;
            for (int j = 0; j < 8; ++j) sum += hist[lane * 8 + j];
            uint32_t incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - sum;
            const unsigned owner = __ballot_sync(0xffffffffu, int64_t(incl) > rank);
            const int first = __ffs(owner) - 1;
            if (lane == first) {
                int64_t cum = excl;
                for (int j = 0; j < 8; ++j) {
                    const uint32_t h = hist[lane * 8 + j];
                    if (cum + h > rank) {
                        s_bucket = uint32_t(lane * 8 + j);
                        s_rank = rank - cum;
                        s_count = h;
                        break;
                    }
                    cum += h;
                }
            }
        }
        __syncthreads();
        prefix |= uint64_t(s_bucket) << shift;
        mask |= uint64_t(0xffu) << shift;
        rank = s_rank;
        if (s_count == 1u) {
            unique = true;
            break;
        }
    }
    uint64_t pivot = prefix;
    if (unique) {
        for (int64_t i = tid; i < c; i += bd) {
            const uint64_t K = composite(i);
            if ((K & mask) == prefix) s_pivot = K;
        }
        __syncthreads();
        pivot = s_pivot;
    }
    if (tid == 0) split[t * (L - 1) + (nodes - 1) + b] = unordered_float(uint32_t(pivot >> 32));

    // ---- stable partition
    const int64_t nl = (c + 1) / 2;
    int64_t lbase = 0, rbase = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = 0; base < c; base += bd) {
        const int64_t i = base + tid;
        const bool valid = i < c;
        int32_t id = 0;
        bool left = false;
        if (valid) {
            id = in[i];
            const uint64_t K = (uint64_t(okey[i]) << 32) | uint32_t(id);
            left = K <= pivot;
        }
        const unsigned lm = __ballot_sync(0xffffffffu, valid && left);
        const unsigned rm = __ballot_sync(0xffffffffu, valid && !left);
        if (lane == 0) {
            s_wl[warp] = __popc(lm);
            s_wr[warp] = __popc(rm);
        }
        __syncthreads();
        // left / right counts of the warps before this one (pl, pr) and of
        // the whole block (tl, tr): an inclusive scan of the per-warp counts
        // across the lanes of every warp
        const uint32_t a = lane < nwarps ? s_wl[lane] : 0u, q = lane < nwarps ? s_wr[lane] : 0u;
        uint32_t ia = a, iq = q;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ya = __shfl_up_sync(0xffffffffu, ia, o);
            const uint32_t yq = __shfl_up_sync(0xffffffffu, iq, o);
            if (lane >= o) {
                ia += ya;
                iq += yq;
            }
        }
        const uint32_t pl = __shfl_sync(0xffffffffu, ia - a, warp);
        const uint32_t pr = __shfl_sync(0xffffffffu, iq - q, warp);
        const uint32_t tl = __shfl_sync(0xffffffffu, ia, 31);
        const uint32_t tr = __shfl_sync(0xffffffffu, iq, 31);
        if (valid) {
            // exactly nl composites are <= pivot (ids are unique), so both
            // destinations stay inside the node's segment; the bounds are
            // checked anyway
            if (left) {
                const int64_t dst = lbase + pl + __popc(lm & lt);
                if (dst < nl) out[dst] = id;
            } else {
                const int64_t dst = nl + rbase + pr + __popc(rm & lt);
                if (dst < c) out[dst] = id;
            }
        }
        lbase += tl;
        rbase += tr;
        __syncthreads();
    }
}

__global__ void k_iota_trees(int32_t *__restrict__ perm, int64_t n, int32_t T) {
    const int64_t total = n * T;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x)
        perm[i] = int32_t(i % n);
}

__global__ void k_leaf_offsets(int32_t *__restrict__ leaf_off, int64_t n, int32_t l) {
    const int64_t L = int64_t(1) << l;
    for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b <= L;
         b += int64_t(gridDim.x) * blockDim.x) {
        if (b == L) {
            leaf_off[b] = int32_t(n);
        } else {
            int64_t off, c;
            node_segment(n, l, b, off, c);
            leaf_off[b] = int32_t(off);
        }
    }
}

// ------------------------------------------------------------- driver ----

namespace {
int pick_rows_per_block(int32_t d) {
    const size_t budget = 160 * 1024;
    for (int rb = 32; rb >= 1; rb >>= 1)
        if (size_t(rb) * size_t(d | 1) * sizeof(float) <= budget) return rb;
    return 0;
}

template <int RB>
cudaError_t launch_project(const mrpt_index *idx, float *Pcm, cudaStream_t s) {
    const size_t smem = size_t(RB) * size_t(idx->d | 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_project_build<RB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    // 32 warps per block: the staged rows allow one or two blocks per SM,
    // and the fmaf chains are latency-bound, so warps are what hides them
    const int64_t blocks = (idx->n + RB - 1) / RB;
    k_project_build<RB><<<dim3(unsigned(blocks)), 1024, smem, s>>>(
        idx->X, idx->n, idx->dpad, idx->d, idx->col_off, idx->dim, idx->val, idx->T * idx->l,
        Pcm);
    return cudaGetLastError();
}
}  // namespace

int grow_trees_device(mrpt_index *idx) {
    cudaStream_t s = idx->stream;
    const int64_t n = idx->n;
    const int32_t T = idx->T, l = idx->l;
    const int64_t L = idx->L;
    int rc;
    int32_t *perm_a = nullptr, *perm_b = nullptr;
    float *Pcm = nullptr;
    const size_t perm_bytes = size_t(T) * size_t(n) * sizeof(int32_t);
    // the leaf array is read in aligned 16-byte groups: 4 spare entries
    const size_t perm_alloc = perm_bytes + 4 * sizeof(int32_t);
    if ((rc = dev_alloc((void **)&perm_a, perm_alloc, "tree permutation"))) return rc;
    {
        const int blocks = int(std::min<int64_t>((int64_t(T) * n + 255) / 256, 152 * 32));
        k_iota_trees<<<blocks, 256, 0, s>>>(perm_a, n, T);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFree(perm_a);
            return cuda_fail(e, "k_iota_trees");
        }
    }
    if (l > 0) {
        const size_t pbytes = size_t(T) * size_t(l) * size_t(n) * sizeof(float);
        if ((rc = dev_alloc((void **)&Pcm, pbytes, "build projections"))) {
            cudaFree(perm_a);
            return rc;
        }
        if ((rc = dev_alloc((void **)&perm_b, perm_alloc, "tree permutation"))) {
            cudaFree(perm_a);
            cudaFree(Pcm);
            return rc;
        }
        uint32_t *okeys = nullptr;
        if ((rc = dev_alloc((void **)&okeys, perm_bytes, "level keys"))) {
            cudaFree(perm_a);
            cudaFree(perm_b);
            cudaFree(Pcm);
            return rc;
        }
        cudaError_t e = cudaSuccess;
        switch (pick_rows_per_block(idx->d)) {
            case 32: e = launch_project<32>(idx, Pcm, s); break;
            case 16: e = launch_project<16>(idx, Pcm, s); break;
            case 8: e = launch_project<8>(idx, Pcm, s); break;
            case 4: e = launch_project<4>(idx, Pcm, s); break;
            case 2: e = launch_project<2>(idx, Pcm, s); break;
            default: e = launch_project<1>(idx, Pcm, s); break;
        }
        const int gblocks = int(std::min<int64_t>((int64_t(T) * n + 255) / 256, 152 * 32));
        for (int32_t j = 0; j < l && e == cudaSuccess; ++j) {
            k_gather_keys<<<gblocks, 256, 0, s>>>(Pcm, n, l, j, T, perm_a, okeys);
            const int64_t blocks = int64_t(T) << j;
            // large nodes (few blocks) get 1,024 threads, small ones 256
            const bool large = (n >> j) >= 16384;
            if (large)
                k_split_level<true><<<dim3(unsigned(blocks)), 1024, 0, s>>>(Pcm, okeys, n, l, j, perm_a, perm_b,
                                                                           idx->split, L);
            else
                k_split_level<false><<<dim3(unsigned(blocks)), 256, 0, s>>>(Pcm, okeys, n, l, j, perm_a, perm_b,
                                                                           idx->split, L);
            e = cudaGetLastError();
            std::swap(perm_a, perm_b);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(okeys);
        cudaFree(Pcm);
        cudaFree(perm_b);
        if (e != cudaSuccess) {
            cudaFree(perm_a);
            return cuda_fail(e, "tree growth kernels");
        }
    }
    idx->leaf_ids = perm_a;
    idx->device_bytes += int64_t(perm_bytes);
    {
        const int blocks = int(std::min<int64_t>((L + 1 + 255) / 256, 152 * 32));
        k_leaf_offsets<<<blocks, 256, 0, s>>>(idx->leaf_off, n, l);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "k_leaf_offsets");
    }
    return MRPT_OK;
}

namespace {

// One thread per entry of the vote layout: entry r of tree t lies in the
// leaf j with 4*off4[j] <= r < 4*off4[j+1] (binary search); it takes the
// leaf's id at that position, or the sentinel past the leaf's end.
__global__ void k_pad_leaves(const int32_t *__restrict__ leaf_ids, int64_t n, int32_t T,
                             const int32_t *__restrict__ leaf_off, const int32_t *__restrict__ off4,
                             int64_t L, int64_t s4, int32_t sentinel, int32_t *__restrict__ out) {
    const int64_t per_tree = 4 * s4;
    const int64_t total = int64_t(T) * per_tree;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = e / per_tree;
        const int64_t r = e - t * per_tree;
        int64_t lo = 0, hi = L;  // last leaf j with 4*off4[j] <= r
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (4 * int64_t(off4[mid]) <= r)
                lo = mid;
            else
                hi = mid;
        }
        const int64_t pos = r - 4 * int64_t(off4[lo]);
        const int64_t size = int64_t(leaf_off[lo + 1]) - leaf_off[lo];
        out[e] = pos < size ? leaf_ids[t * n + leaf_off[lo] + pos] : sentinel;
    }
}

// Spreads the entries of each 256-entry window of a padded leaf over counter
// banks.  A warp votes a window with eight shared-memory reductions: lane r
// takes its entries 4r..4r+3 of each 128-entry half h, and reduction (h, u)
// updates window positions 128h + 4r + u for r = 0..31.  Counter bank of id x
// is (x >> 2) mod 32; two lanes of one reduction in the same bank cost an
// extra pass.  Each reduction is therefore given ids of distinct banks while
// it can, always from the banks with the most entries left (so that the
// crowded banks spread over all eight).  Votes do not depend on the order, so
// only the layout changes.  One thread per window; build-time only.
__global__ void k_bank_spread_windows(int32_t *__restrict__ leaf4, int32_t T,
                                      const int32_t *__restrict__ off4, int64_t L, int64_t s4,
                                      int32_t win) {
    const int64_t total = int64_t(T) * L * win;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = g / (L * win);
        const int64_t r0 = g - t * L * win;
        const int64_t j = r0 / win;
        const int32_t w = int32_t(r0 - j * win);
        const int32_t len4 = off4[j + 1] - off4[j];
        if (64 * w >= len4) continue;
        const int32_t n4 = min(64, len4 - 64 * w);
        int32_t *base = leaf4 + 4 * (t * s4 + off4[j] + 64 * int64_t(w));
        int32_t byb[256];   // entries grouped by bank
        int32_t start[33];
        int32_t rem[32];
        for (int b = 0; b <= 32; ++b) start[b] = 0;
        for (int e = 0; e < 4 * n4; ++e) ++start[((base[e] >> 2) & 31) + 1];
        for (int b = 0; b < 32; ++b) start[b + 1] += start[b];
        for (int b = 0; b < 32; ++b) rem[b] = start[b + 1] - start[b];
        {
            int32_t fill[32];
            for (int b = 0; b < 32; ++b) fill[b] = start[b];
            for (int e = 0; e < 4 * n4; ++e) {
                const int32_t x = base[e];
                byb[fill[(x >> 2) & 31]++] = x;
            }
        }
        for (int h = 0; h < 2; ++h) {
            const int cap = max(0, min(32, n4 - 32 * h));
            for (int u = 0; u < 4; ++u) {
                uint32_t used = 0u;
                for (int r = 0; r < cap; ++r) {
                    int best = -1, best_any = -1;
                    for (int b = 0; b < 32; ++b) {
                        if (rem[b] == 0) continue;
                        if (best_any < 0 || rem[b] > rem[best_any]) best_any = b;
                        if (!((used >> b) & 1u) && (best < 0 || rem[b] > rem[best])) best = b;
                    }
                    const int b = best >= 0 ? best : best_any;
                    --rem[b];
                    used |= 1u << b;
                    base[128 * h + 4 * r + u] = byb[start[b] + rem[b]];
                }
            }
        }
    }
}

}  // namespace

// Position of the first id >= c * VOTE_CHUNK_IDS in every leaf of every
// tree (the leaf's ids ascend), for c = 0 .. C: one thread per (tree, leaf,
// c), a binary search over the leaf.
__global__ void k_chunk_bounds(const int32_t *__restrict__ leaf_ids, int64_t n, int32_t T,
                               const int32_t *__restrict__ leaf_off, int64_t L, int32_t C,
                               int32_t *__restrict__ bnd) {
    const int64_t total = int64_t(T) * L * (C + 1);
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total;
         x += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = int32_t(x % (C + 1));
        const int64_t tj = x / (C + 1);
        const int64_t j = tj % L;
        const int64_t t = tj / L;
        int32_t lo = leaf_off[j], hi = leaf_off[j + 1];
        const int32_t *ids = leaf_ids + t * n;
        const int64_t lim = int64_t(c) * VOTE_CHUNK_IDS;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (int64_t(ids[mid]) < lim)
                lo = mid + 1;
            else
                hi = mid;
        }
        bnd[x] = lo;
    }
}

int build_vote_layout(mrpt_index *idx) {
    if (idx->n > VOTE_CHUNK_IDS) {
        const int32_t C = int32_t((idx->n + VOTE_CHUNK_IDS - 1) / VOTE_CHUNK_IDS);
        const int64_t total = int64_t(idx->T) * idx->L * (C + 1);
        int rc;
        if ((rc = dev_alloc((void **)&idx->chunk_bnd, size_t(total) * 4, "id-chunk bounds"))) return rc;
        idx->device_bytes += total * 4;
        idx->n_chunks = C;
        const int blocks = int(std::min<int64_t>((total + 255) / 256, 152 * 32));
        k_chunk_bounds<<<blocks, 256, 0, idx->stream>>>(idx->leaf_ids, idx->n, idx->T, idx->leaf_off, idx->L, C,
                                                        idx->chunk_bnd);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "k_chunk_bounds");
        return MRPT_OK;
    }
    const int64_t L = idx->L;
    std::vector<int32_t> off(size_t(L + 1)), off4(size_t(L + 1));
    cudaError_t e = cudaMemcpy(off.data(), idx->leaf_off, size_t(L + 1) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "vote layout: leaf offsets");
    int32_t longest = 0;
    off4[0] = 0;
    for (int64_t j = 0; j < L; ++j) {
        const int32_t len4 = (off[size_t(j + 1)] - off[size_t(j)] + 3) / 4;
        off4[size_t(j + 1)] = off4[size_t(j)] + len4;
        longest = std::max(longest, len4);
    }
    const int64_t s4 = off4[size_t(L)];
    const size_t bytes = size_t(idx->T) * size_t(s4 > 0 ? s4 : 1) * 16;
    int rc;
    if ((rc = dev_alloc((void **)&idx->leaf_off4, size_t(L + 1) * 4, "vote layout offsets"))) return rc;
    if ((rc = dev_alloc((void **)&idx->leaf4, bytes, "vote layout"))) return rc;
    idx->device_bytes += int64_t(bytes + size_t(L + 1) * 4);
    idx->vote_s4 = s4;
    idx->vote_win = (longest + 31) / 32;
    e = cudaMemcpy(idx->leaf_off4, off4.data(), size_t(L + 1) * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "vote layout: offsets upload");
    const int64_t total = int64_t(idx->T) * 4 * s4;
    if (total > 0) {
        const int blocks = int(std::min<int64_t>((total + 255) / 256, 152 * 32));
        k_pad_leaves<<<blocks, 256, 0, idx->stream>>>(idx->leaf_ids, idx->n, idx->T, idx->leaf_off,
                                                       idx->leaf_off4, L, s4, vote_sentinel(idx->n),
                                                       reinterpret_cast<int32_t *>(idx->leaf4));
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const int32_t win256 = (idx->vote_win + 1) / 2;
            const int64_t windows = int64_t(idx->T) * L * win256;
            const int wblocks = int(std::min<int64_t>((windows + 127) / 128, 152 * 16));
            k_bank_spread_windows<<<wblocks, 128, 0, idx->stream>>>(reinterpret_cast<int32_t *>(idx->leaf4),
                                                                   idx->T, idx->leaf_off4, L, s4, win256);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "k_pad_leaves");
    }
    return MRPT_OK;
}

// Leaf offsets of a loaded index (they depend only on n and l).
int compute_leaf_offsets(mrpt_index *idx) {
    const int blocks = int(std::min<int64_t>((idx->L + 1 + 255) / 256, 152 * 32));
    k_leaf_offsets<<<blocks, 256, 0, idx->stream>>>(idx->leaf_off, idx->n, idx->l);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "k_leaf_offsets");
    return MRPT_OK;
}

}  // namespace mrpt
