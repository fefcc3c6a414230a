// Top-k merge of per-shard results (the exchange step of a row-sharded
// search) and of per-basis results (multi-basis search, where one point can
// come from several lists and counts once).  Cone keys depend only on a row,
// so a shard holding rows [lo, hi) builds exactly the part of every cone that
// falls in its rows, and a query probes the same cones on every shard; the
// union of the shards' candidates is the unsharded candidate set, and the k
// best of the shards' k-best lists (by distance, then global id) are the
// unsharded answer, bit for bit (a pair's distance does not depend on the
// sharding).
#include "osann.h"
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

// One warp per query: the G lists of k (distance, id) pairs of that query,
// packed as (distance bits, id) so that the u64 order is (distance, id).
template <int KMAX>
__global__ void __launch_bounds__(128) merge_lists_kernel(const int64_t* __restrict__ ids, const float* __restrict__ d2,
                                                          int G, int64_t Q, int k, int64_t* __restrict__ out_ids,
                                                          float* __restrict__ out_d)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    uint64_t list[KMAX];
    topk_init<KMAX>(list, k);
    const int64_t n = int64_t(G) * k;
    for (int64_t j = lane; j < n; j += 32) {
        const int64_t g = j / k, r = j % k;
        const int64_t at = (g * Q + q) * k + r;
        const int64_t id = ids[at];
        if (id < 0) continue;  // padding
        const uint64_t v = pack_di(d2[at], uint32_t(id));
        if (v < list[KMAX - 1]) {
            // the same point from another list (another basis) is one candidate;
            // copies held by other lanes leave together when extracted below
            bool dup = false;
#pragma unroll
            for (int u = 0; u < KMAX; ++u) dup |= u >= KMAX - k && list[u] == v;  // live slots only
            if (!dup) topk_insert<KMAX>(list, v);
        }
    }
    for (int j = 0; j < k; ++j) {
        const uint64_t head = topk_head<KMAX>(list, k);
        const uint64_t best = warp_min_u64(head);
        if (head == best && best != EMPTY_DI) topk_remove<KMAX>(list, k, best);
        if (lane == 0) {
            const uint32_t id = di_id(best);
            out_ids[q * k + j] = best == EMPTY_DI ? int64_t(-1) : int64_t(id);
            out_d[q * k + j] = best == EMPTY_DI ? INFINITY : di_dist(best);
        }
    }
}

}  // namespace osann

using namespace osann;

extern "C" int osann_merge_topk(const int64_t* d_ids, const float* d_sqdists, int32_t G, int64_t Q, int32_t k,
                                int64_t* d_out_ids, float* d_out_sqdists, void* stream)
{
    if (G < 1 || Q < 0 || k < 1 || k > MAX_K || (Q > 0 && (!d_ids || !d_sqdists || !d_out_ids || !d_out_sqdists))) {
        set_error("osann_merge_topk: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    if (Q == 0) return OSANN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = unsigned((Q + 3) / 4);
#define OSANN_MERGE(KM) merge_lists_kernel<KM><<<blocks, 128, 0, st>>>(d_ids, d_sqdists, G, Q, k, d_out_ids, d_out_sqdists)
    if (k <= 1) OSANN_MERGE(1);
    else if (k <= 4) OSANN_MERGE(4);
    else if (k <= 16) OSANN_MERGE(16);
    else OSANN_MERGE(32);
#undef OSANN_MERGE
    return count_launch();
}
