// osann_search_noalloc: the plain search with its scratch memory in a
// file-scope device array instead of a caller- or library-allocated
// workspace, for callers that cannot allocate device memory when they
// query (see the declaration in include/osann.h).
//
// The array is part of this library's device image: every GPU that loads
// the library holds it until the process exits.  Host code must not pass
// the array's name to a kernel (on the host it is only a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

#include "osann.h"
#include "osann_launch.h"

namespace osann {
int index_device(const osann_index* ix);
}

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_addr[64];

// The scratch array of the current device, which must be the index's: the
// array of another device would put the kernels' scratch on that device.
int scratch_address(int index_dev, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        osann::set_error("osann_search_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return OSANN_ERR_CUDA;
    }
    if (dev != index_dev) {
        osann::set_error("osann_search_noalloc: the current device (%d) is not the index's device (%d)", dev,
                         index_dev);
        return OSANN_ERR_INVALID;
    }
    if (dev < 0 || dev >= 64) {
        osann::set_error("osann_search_noalloc: device ordinal %d out of range", dev);
        return OSANN_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // with `dev` current
        if (e != cudaSuccess || !p) {
            osann::set_error("osann_search_noalloc: scratch address lookup failed: %s", cudaGetErrorString(e));
            return OSANN_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return OSANN_OK;
}

}  // namespace

extern "C" int osann_search_noalloc(const osann_index* index, const float* d_queries, int64_t Q, int32_t P,
                                    int32_t k, int64_t* d_ids, float* d_sqdists, void* stream)
{
    if (!index || Q < 0 || P < 1 || k < 1 || k > 32) {
        osann::set_error("osann_search_noalloc: invalid arguments (Q=%lld P=%d k=%d)", (long long)Q, P, k);
        return OSANN_ERR_INVALID;
    }
    const size_t need = osann_search_workspace_size(index, Q, P, k, OSANN_PATH_PLAIN);
    if (need == 0 || need > NOALLOC_SCRATCH_BYTES) {
        osann::set_error("osann_search_noalloc: needs %zu bytes of scratch, above the fixed %zu-byte maximum "
                         "(use fewer queries per call or osann_search)",
                         need, NOALLOC_SCRATCH_BYTES);
        return OSANN_ERR_INVALID;
    }
    void* scratch = nullptr;
    int rc = scratch_address(osann::index_device(index), &scratch);
    if (rc) return rc;
    // every scratch byte the plain path reads is written earlier in the same
    // call, so nothing needs clearing between calls
    return osann_search(index, d_queries, Q, P, k, OSANN_PATH_PLAIN, scratch, NOALLOC_SCRATCH_BYTES, d_ids, d_sqdists,
                        stream);
}
