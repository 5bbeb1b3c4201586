// mrpt_query_noalloc: the query without any device allocation.
//
// mrpt_query keeps its scratch (the leaf of every query in every tree, and
// the counter that hands queries to blocks) in buffers that the index grows
// with cudaMalloc on first use.  Some callers cannot allow that: a serving
// loop with a latency budget (cudaMalloc/cudaFree can synchronise the whole
// device), or a process whose device memory is owned by another framework's
// pool or capped by it.  This entry point runs the same kernels with that
// scratch in a fixed array of this file instead; the caller passes device
// buffers for the inputs and outputs, as always.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "mrpt_internal.cuh"

namespace mrpt {
namespace {

// 4 MiB, held on every device that loads the library until the process
// exits: 64 words (256 bytes) of header -- word 0 is the work counter --
// then the leaf-of-query table (m x n_trees int32).
constexpr size_t kScratchWords = size_t(1) << 20;
constexpr size_t kHeaderWords = 64;
static_assert(MRPT_NOALLOC_MAX_LEAF_ENTRIES == kScratchWords - kHeaderWords,
              "header constant out of date");

static __device__ __align__(256) uint32_t g_scratch[kScratchWords];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
uint32_t *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on `dev` (which must be current).  In host
// code `g_scratch` names a host-side stand-in, so the address is asked of
// the runtime once per device and kept.
int scratch_on(int dev, uint32_t **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("mrpt_query_noalloc: device ordinal out of range");
        return MRPT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "mrpt_query_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_addr[dev];
    return MRPT_OK;
}

}  // namespace
}  // namespace mrpt

using namespace mrpt;

extern "C" int mrpt_query_noalloc(mrpt_index *idx, const float *Q, int64_t m, int32_t k,
                                  int32_t v, int32_t n_trees, int32_t *out_ids,
                                  float *out_dists) {
    clear_error();
    if (!idx) {
        set_error("mrpt_query_noalloc: idx is NULL");
        return MRPT_ERR_INVALID_ARG;
    }
    const int32_t T_use = n_trees > 0 ? n_trees : idx->T;
    if (m < 0 || (m > 0 && (!Q || !out_ids || !out_dists)) || k < 1 || k > MRPT_MAX_K ||
        v < 1 || T_use > idx->T || v > T_use) {
        set_error("mrpt_query_noalloc: invalid argument (need m >= 0, non-NULL buffers, 1 <= k <= " +
                  std::to_string(MRPT_MAX_K) + ", 1 <= v <= n_trees <= T)");
        return MRPT_ERR_INVALID_ARG;
    }
    if (m == 0) return MRPT_OK;
    if (m > int64_t(MRPT_NOALLOC_MAX_LEAF_ENTRIES) / T_use) {
        set_error("mrpt_query_noalloc: m * n_trees = " + std::to_string(m) + " * " +
                  std::to_string(T_use) + " exceeds the fixed scratch of " +
                  std::to_string(MRPT_NOALLOC_MAX_LEAF_ENTRIES) + " entries; split the batch");
        return MRPT_ERR_INVALID_ARG;
    }
    if (!is_device_ptr(Q) || !is_device_ptr(out_ids) || !is_device_ptr(out_dists)) {
        set_error("mrpt_query_noalloc: Q, out_ids and out_dists must be device memory");
        return MRPT_ERR_INVALID_ARG;
    }
    int dev = -1;
    MRPT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != idx->device) {
        set_error("mrpt_query_noalloc: the index lives on device " + std::to_string(idx->device) +
                  " but device " + std::to_string(dev) + " is current");
        return MRPT_ERR_INVALID_ARG;
    }
    uint32_t *scratch = nullptr;
    int rc = scratch_on(dev, &scratch);
    if (rc) return rc;

    QueryLaunch ql{};
    ql.Q = Q;
    ql.m = m;
    ql.k = k;
    ql.v = v;
    ql.n_trees = T_use;
    ql.out_ids = out_ids;
    ql.out_dists = out_dists;
    ql.leaf = reinterpret_cast<int32_t *>(scratch + kHeaderWords);
    return launch_query_with_counter(idx, ql, scratch);
}
