// Second-level cone table (Sec. 4: an extra hash level over the per-basis
// tables once the cone count is too large for a direct table).
//
// With N_C >= 2^31 the direct CSR over all N_C cones cannot be allocated, but
// at most min(N, N_C) cones hold a point.  The build sorts the point ids by
// their 128-bit cone id (launch_stable_sort_wide), then here:
//   - the heads of equal-id runs give the occupied cones, numbered 0..n_occ-1
//     in ascending id order ("compact" cones);
//   - offsets[] is the CSR over NCt = min(N, N_C) + 1 compact cones, those
//     from n_occ on empty (so compact cone NCt - 1 is always empty and serves
//     as the image of every probed id that no point carries);
//   - ukeys[c] is the 128-bit id of compact cone c;
//   - an open-addressing hash table (linear probing, capacity a power of two
//     at least 2 NCt) maps a 128-bit id to its compact cone.
// Everything after the probe lists (work list, scans, screening, rerank)
// sees compact cones only and is unchanged.  Nothing here waits on another
// block; the only loop, the insertion's probe sequence, is bounded by the
// table size and ends early because the table is at most half full.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

__global__ void __launch_bounds__(256) run_heads_kernel(const uint4* __restrict__ wkeys,
                                                        const uint32_t* __restrict__ perm, int64_t N,
                                                        uint32_t* __restrict__ heads)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
        heads[i] = (i == 0 || !wide_eq(wkeys[perm[i]], wkeys[perm[i - 1]])) ? 1u : 0u;
}

// ex = exclusive scan of heads: sorted position i lies in compact cone
// ex[i] + heads[i] - 1.
__global__ void __launch_bounds__(256) cone_table_kernel(const uint4* __restrict__ wkeys,
                                                         const uint32_t* __restrict__ perm,
                                                         const uint32_t* __restrict__ heads,
                                                         const uint32_t* __restrict__ ex, int64_t N, int64_t NCt,
                                                         uint32_t* __restrict__ keys, uint32_t* __restrict__ offsets,
                                                         uint4* __restrict__ ukeys, uint32_t* __restrict__ n_occ)
{
    const uint32_t nocc = ex[N - 1] + heads[N - 1];
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t span = N > NCt + 1 ? N : NCt + 1;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < span; i += stride) {
        if (i < N) {
            const uint32_t h = heads[i];
            const uint32_t c = ex[i] + h - 1u;
            const uint32_t id = perm[i];
            keys[id] = c;
            if (h) {
                offsets[c] = uint32_t(i);
                ukeys[c] = wkeys[id];
            }
        }
        if (i >= int64_t(nocc) && i <= NCt) {
            offsets[i] = uint32_t(N);
            if (i < NCt) ukeys[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_occ = nocc;
}

__global__ void __launch_bounds__(256) hash_insert_kernel(const uint4* __restrict__ ukeys,
                                                          const uint32_t* __restrict__ n_occ,
                                                          uint32_t* __restrict__ htab, uint32_t hmask)
{
    const uint32_t n = *n_occ;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        uint32_t h = cone_hash(ukeys[c]) & hmask;
        for (uint32_t it = 0; it <= hmask; ++it) {
            if (atomicCAS(htab + h, HASH_EMPTY, c) == HASH_EMPTY) break;
            h = (h + 1) & hmask;
        }
    }
}

size_t cone_table_temp_bytes(int64_t N)
{
    const size_t nb = size_t((N + 63) / 64 * 64) * 4;
    return 2 * nb + (scan_temp_bytes(N) + 255) / 256 * 256 + 256;
}

int launch_cone_table(const uint4* wkeys, const uint32_t* perm, int64_t N, int64_t NCt, uint32_t* keys,
                      uint32_t* offsets, uint4* ukeys, uint32_t* n_occ, uint32_t* htab, uint32_t hmask, void* temp,
                      cudaStream_t st, int num_sms)
{
    if (N < 1 || NCt < 1) return -1;
    const size_t nb = size_t((N + 63) / 64 * 64) * 4;
    char* t = static_cast<char*>(temp);
    uint32_t* heads = reinterpret_cast<uint32_t*>(t);
    uint32_t* ex = reinterpret_cast<uint32_t*>(t + nb);
    void* stemp = t + 2 * nb;
    const int64_t cap = int64_t(num_sms) * 8;
    int64_t blocks = (N + 255) / 256;
    if (blocks > cap) blocks = cap;
    run_heads_kernel<<<unsigned(blocks), 256, 0, st>>>(wkeys, perm, N, heads);
    int rc = count_launch();
    if (!rc) rc = launch_exclusive_scan(heads, ex, N, stemp, st);
    if (rc) return rc;
    const int64_t span = N > NCt + 1 ? N : NCt + 1;
    blocks = (span + 255) / 256;
    if (blocks > cap) blocks = cap;
    cone_table_kernel<<<unsigned(blocks), 256, 0, st>>>(wkeys, perm, heads, ex, N, NCt, keys, offsets, ukeys, n_occ);
    rc = count_launch();
    if (rc) return rc;
    if (cudaMemsetAsync(htab, 0xFF, (size_t(hmask) + 1) * 4, st) != cudaSuccess) return -5;
    blocks = (NCt + 255) / 256;
    if (blocks > cap) blocks = cap;
    hash_insert_kernel<<<unsigned(blocks), 256, 0, st>>>(ukeys, n_occ, htab, hmask);
    return count_launch();
}

}  // namespace osann
