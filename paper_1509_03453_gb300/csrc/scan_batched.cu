// Batched candidate scan: the (query, probed cone) pairs of a whole query
// batch are inverted into cone-major work, so that each cone's points are
// streamed once per group of queries that visit it instead of once per query.
// The arithmetic per (query, point) pair is exactly the plain scan's (fp32
// direct differences, Eq. 1), so results are identical to the plain path.
//
//   work list  (all on device, no host round trip, graph-capturable):
//     qcount[c]  = number of queries that probe non-empty cone c
//     qoff       = exclusive scan of qcount
//     qlist      = the (query, probe position) slots q * P + p grouped by cone
//                  (ascending inside a cone's run of each block's chunk)
//     items      = (cone, group) pairs, group = up to G consecutive slots of
//                  the cone's list; G = 128 / TPR queries per CTA
//   tile scan  (persistent CTAs, atomic work counter):
//     thread 0 streams the rows of successive items into a ring of shared
//     memory stages with 1-D bulk copies (TMA engine) and mbarriers, across
//     item boundaries; every thread owns one query slice (DPT dims of one
//     query, TPR threads per query) and compares it with every row of the
//     stage (broadcast reads); a register top-k per query is flushed to the
//     query's slot when the item ends.
//   merge      (one warp per query): top-k over the query's slots.
//
// Linear search (Eq. 1 over all N) reuses the tile scan in a dense mode:
// items are (row chunk, consecutive query group) pairs.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

constexpr int TILE_THREADS = 128;
constexpr int TILE_STAGES = 4;
constexpr int TILE_STAGE_FLOATS = 4096;  // 16 KB per stage
constexpr int BF_CHUNK_ROWS = 4096;      // rows per linear-search chunk

// ---------------------------------------------------------------- work list

// probe values are < N_C by construction; the bound check guards the reads
__device__ __forceinline__ bool cone_nonempty(const uint32_t* __restrict__ offsets, uint32_t b, uint32_t NC)
{
    return b < NC && __ldg(offsets + b + 1) > __ldg(offsets + b);
}

__global__ void wl_count_global_kernel(const uint32_t* __restrict__ probes, int64_t n,
                                       const uint32_t* __restrict__ offsets, uint32_t NC,
                                       uint32_t* __restrict__ qcount)
{
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t b = probes[t];  // order does not matter for counting
        if (cone_nonempty(offsets, b, NC)) atomicAdd(&qcount[b], 1u);
    }
}

__global__ void wl_fill_kernel(const uint32_t* __restrict__ probes, int64_t n, const uint32_t* __restrict__ offsets,
                               uint32_t NC, const uint32_t* __restrict__ qoff, uint32_t* __restrict__ fill,
                               uint32_t* __restrict__ qlist)
{
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t b = probes[t];
        if (cone_nonempty(offsets, b, NC)) qlist[qoff[b] + atomicAdd(&fill[b], 1u)] = uint32_t(t);
    }
}

// Shared-memory bitmap of the non-empty cones (N_C <= 12288), one ballot per
// 32 cones of the offsets; ends with a block barrier.
__device__ __forceinline__ void load_nonempty_bits(const uint32_t* __restrict__ offsets, int NC,
                                                   uint32_t* __restrict__ bits)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 32 * warp; c0 < NC; c0 += 32 * nw) {
        const int c = c0 + lane;
        const bool ne = c < NC && __ldg(offsets + c + 1) > __ldg(offsets + c);
        const uint32_t m = __ballot_sync(0xffffffffu, ne);
        if (lane == 0) bits[c0 >> 5] = m;
    }
    __syncthreads();
}

__device__ __forceinline__ bool bit_nonempty(const uint32_t* __restrict__ bits, uint32_t b, uint32_t NC)
{
    return b < NC && ((bits[b >> 5] >> (b & 31)) & 1u);
}

// Calls f(t, cone) for every probe t of [t0, t1), four per thread per step
// (t0 a multiple of 4; the probe array 16-byte aligned).
template <typename F>
__device__ __forceinline__ void for_chunk_probes(const uint32_t* __restrict__ probes, int64_t t0, int64_t t1, F f)
{
    const uint4* p4 = reinterpret_cast<const uint4*>(probes);
    const int64_t v1 = t1 >> 2;
    for (int64_t v = (t0 >> 2) + threadIdx.x; v < v1; v += blockDim.x) {
        const uint4 b = p4[v];
        f(4 * v, b.x);
        f(4 * v + 1, b.y);
        f(4 * v + 2, b.z);
        f(4 * v + 3, b.w);
    }
    for (int64_t t = 4 * v1 + threadIdx.x; t < t1; t += blockDim.x) f(t, probes[t]);
}

// Cone-major per-block histograms: H[c * nb + b] = probes of block b's chunk
// that hit non-empty cone c.  One exclusive scan of H (plus a trailing zero)
// then gives every (cone, block) its first slot in the cone-major list.
// Shared memory: N_C counters and the N_C-bit non-empty bitmap.
__global__ void __launch_bounds__(512) wl_block_hist_kernel(const uint32_t* __restrict__ probes, int64_t n,
                                                            int64_t chunk, const uint32_t* __restrict__ offsets,
                                                            int NC, uint32_t* __restrict__ H)
{
    extern __shared__ uint32_t h[];
    uint32_t* bits = h + NC;
    for (int c = threadIdx.x; c < NC; c += blockDim.x) h[c] = 0;
    load_nonempty_bits(offsets, NC, bits);
    const int64_t t0 = int64_t(blockIdx.x) * chunk, t1 = t0 + chunk < n ? t0 + chunk : n;
    for_chunk_probes(probes, t0, t1, [&](int64_t, uint32_t b) {
        if (bit_nonempty(bits, b, uint32_t(NC))) atomicAdd(&h[b], 1u);
    });
    __syncthreads();
    for (int c = threadIdx.x; c < NC; c += blockDim.x) H[int64_t(c) * gridDim.x + blockIdx.x] = h[c];
}

// Also writes the item descriptors (first row, end row, first slot, slot
// count) of the cones c = blockIdx.x + j * gridDim.x, from the per-cone
// counts, first slots and item offsets of wl_cones_kernel.
__global__ void __launch_bounds__(512) wl_block_fill_kernel(const uint32_t* __restrict__ probes, int64_t n,
                                                            int64_t chunk, const uint32_t* __restrict__ offsets,
                                                            int NC, const uint32_t* __restrict__ Hs,
                                                            uint32_t* __restrict__ qlist,
                                                            const uint32_t* __restrict__ qcount,
                                                            const uint32_t* __restrict__ qoff,
                                                            const uint32_t* __restrict__ item_off, int G,
                                                            uint4* __restrict__ items)
{
    extern __shared__ uint32_t cur[];
    uint32_t* bits = cur + NC;
    for (int c = threadIdx.x; c < NC; c += blockDim.x) cur[c] = Hs[int64_t(c) * gridDim.x + blockIdx.x];
    // this block's share of the item descriptors: one warp per cone
    for (int c = int(blockIdx.x) + int(gridDim.x) * int(threadIdx.x >> 5); c < NC;
         c += int(gridDim.x) * int(blockDim.x >> 5)) {
        const uint32_t cnt = qcount[c], o = item_off[c], ni = (cnt + uint32_t(G) - 1) / uint32_t(G);
        const uint32_t r0 = offsets[c], r1 = offsets[c + 1], q0 = qoff[c];
        for (uint32_t g = threadIdx.x & 31; g < ni; g += 32) {
            const uint32_t rest = cnt - g * uint32_t(G);
            items[o + g] = make_uint4(r0, r1, q0 + g * uint32_t(G), rest < uint32_t(G) ? rest : uint32_t(G));
        }
    }
    load_nonempty_bits(offsets, NC, bits);  // (its barrier also publishes cur)
    const int64_t t0 = int64_t(blockIdx.x) * chunk, t1 = t0 + chunk < n ? t0 + chunk : n;
    for_chunk_probes(probes, t0, t1, [&](int64_t t, uint32_t b) {
        if (bit_nonempty(bits, b, uint32_t(NC))) qlist[atomicAdd(&cur[b], 1u)] = uint32_t(t);
    });
}

__global__ void wl_nitems_kernel(const uint32_t* __restrict__ qcount, int64_t NC, int G, uint32_t* __restrict__ nitems)
{
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c <= NC; c += int64_t(gridDim.x) * blockDim.x)
        nitems[c] = c < NC ? (qcount[c] + G - 1) / G : 0u;
}

// Item descriptors (first row, end row, first slot, slot count) of every
// (cone, query group) pair.
__global__ void wl_items_kernel(const uint32_t* __restrict__ nitems, const uint32_t* __restrict__ item_off,
                                const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ qcount,
                                const uint32_t* __restrict__ qoff, int64_t NC, int G, uint4* __restrict__ items,
                                uint32_t* __restrict__ counters)
{
    const int64_t gtid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (gtid == 0) counters[0] = 0;  // work counter of the tile scan that follows
    for (int64_t c = gtid; c < NC; c += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t n = nitems[c], o = item_off[c];
        if (n == 0) continue;
        const uint32_t r0 = offsets[c], r1 = offsets[c + 1], cnt = qcount[c], q0 = qoff[c];
        for (uint32_t g = 0; g < n; ++g) {
            const uint32_t rest = cnt - g * uint32_t(G);
            items[o + g] = make_uint4(r0, r1, q0 + g * uint32_t(G), rest < uint32_t(G) ? rest : uint32_t(G));
        }
    }
}

// One CTA over all cones (N_C <= 12288, at most 12 per thread): per-cone
// counts and first slots from the scanned per-block histograms, the number of
// items of each cone and their exclusive scan, in one launch (the many-block
// fill kernel then writes the item descriptors).  item_off[N_C] receives the
// total.
constexpr int WL_CONES_THREADS = 1024;
constexpr int WL_CONES_PER = 12;  // cones per thread: N_C <= 12 * 1024

__global__ void __launch_bounds__(WL_CONES_THREADS) wl_cones_kernel(
    const uint32_t* __restrict__ Hs, int NC, int64_t nb, int G, uint32_t* __restrict__ qcount,
    uint32_t* __restrict__ qoff, uint32_t* __restrict__ item_off, uint32_t* __restrict__ counters)
{
    __shared__ uint32_t wsum[WL_CONES_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (NC + WL_CONES_THREADS - 1) / WL_CONES_THREADS;  // <= WL_CONES_PER
    const int c0 = tid * per < NC ? tid * per : NC, c1 = c0 + per < NC ? c0 + per : NC;
    // this thread's cone boundaries in the scanned histogram (Hs[N_C * nb] is the
    // total), all loads in flight at once
    uint32_t e[WL_CONES_PER + 1];
#pragma unroll
    for (int i = 0; i <= WL_CONES_PER; ++i) e[i] = c0 + i <= c1 ? Hs[int64_t(c0 + i) * nb] : 0u;
    uint32_t mine = 0, ni[WL_CONES_PER];
#pragma unroll
    for (int i = 0; i < WL_CONES_PER; ++i) {
        ni[i] = 0;
        if (c0 + i < c1) {
            const uint32_t cnt = e[i + 1] - e[i];
            qoff[c0 + i] = e[i];
            qcount[c0 + i] = cnt;
            ni[i] = (cnt + uint32_t(G) - 1) / uint32_t(G);
            mine += ni[i];
        }
    }
    // exclusive scan of the per-thread item counts over the CTA
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        wsum[lane] = wi - w;  // exclusive over warps
    }
    __syncthreads();
    uint32_t off = wsum[warp] + incl - mine;
#pragma unroll
    for (int i = 0; i < WL_CONES_PER; ++i)
        if (c0 + i < c1) {
            item_off[c0 + i] = off;
            off += ni[i];
        }
    if (tid == WL_CONES_THREADS - 1) item_off[NC] = off;
    if (tid == 0) counters[0] = 0;  // work counter of the scan that follows
}

static int wl_blocks_impl(int64_t n, int num_sms)
{
    int64_t nb = (n + 4095) / 4096;
    if (nb > 2 * num_sms) nb = 2 * num_sms;
    return int(nb < 1 ? 1 : nb);
}

int wl_hist_entries(int64_t NC, int64_t n, int num_sms)
{
    return NC <= 12288 ? int(NC * wl_blocks_impl(n, num_sms) + 1) : 0;
}

size_t batched_scan_temp_bytes(int64_t NC, int64_t n, int num_sms)
{
    const int64_t hn = NC <= 12288 ? NC * wl_blocks_impl(n, num_sms) + 1 : 0;
    int64_t m = hn > NC + 1 ? hn : NC + 1;
    return scan_temp_bytes(m);
}


// ---------------------------------------------------------------- query-set work list
//
// For the tensor-core screen only the query of a slot matters, so its lists
// can be built from query sets instead of inverting every (query, position)
// slot with a scattered store: B[c * W + w] (W = ceil(Q / 32)) holds, in bit
// j, whether query 32 w + j probes non-empty cone c.  Blocks of 32 queries OR
// their bits into shared memory; a warp per cone then counts its bits, and
// after one scan over the cones expands them in ascending query order into
// contiguous runs of qlist (entry q * S, so entry / S is the query).

constexpr int QSET_THREADS = 256;
constexpr int QSET_PCHUNK = 4 * QSET_THREADS;  // slots of a query per block: four per thread

// Block (w, part): queries 32 w .. 32 w + 31, slots [part * QSET_PCHUNK, ...)
// of each (S slots per query; a 16-byte load per query row and thread when
// S % 4 == 0, eight rows in flight).  B must be zero on entry.
__global__ void __launch_bounds__(QSET_THREADS) wl_qset_kernel(const uint32_t* __restrict__ probes, int64_t Q,
                                                               int64_t S, const uint32_t* __restrict__ offsets,
                                                               int NC, int64_t W, uint32_t* __restrict__ B)
{
    extern __shared__ uint32_t qs_words[];
    uint32_t* bits = qs_words + NC;
    for (int c = threadIdx.x; c < NC; c += blockDim.x) qs_words[c] = 0;
    load_nonempty_bits(offsets, NC, bits);
    const int64_t q0 = int64_t(blockIdx.x) * 32;
    const int nq = int(Q - q0 < 32 ? Q - q0 : 32);
    // the block's slot range holds nv groups of four; with nv < blockDim the
    // threads take several rows at once (row j0, j0 + jstep, ...)
    const int64_t pb = int64_t(blockIdx.y) * QSET_PCHUNK, pe = pb + QSET_PCHUNK < S ? pb + QSET_PCHUNK : S;
    const int nv = int((pe - pb + 3) / 4), jstep = int(blockDim.x) / nv;
    const int j0 = int(threadIdx.x) / nv;
    const int64_t p = pb + 4 * int64_t(threadIdx.x % nv);  // this thread's slots
    auto set = [&](uint32_t c, int j) {
        if (bit_nonempty(bits, c, uint32_t(NC))) atomicOr(&qs_words[c], 1u << j);
    };
    if (j0 < jstep) {
        if ((S & 3) == 0) {
#pragma unroll 8
            for (int j = j0; j < nq; j += jstep) {
                const uint4 c = *reinterpret_cast<const uint4*>(probes + (q0 + j) * S + p);
                set(c.x, j);
                set(c.y, j);
                set(c.z, j);
                set(c.w, j);
            }
        } else {
            for (int j = j0; j < nq; j += jstep)
                for (int i = 0; i < 4; ++i)
                    if (p + i < pe) set(probes[(q0 + j) * S + p + i], j);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NC; c += blockDim.x) {
        const uint32_t m = qs_words[c];
        if (m) atomicOr(&B[int64_t(c) * W + blockIdx.x], m);
    }
}

// Warp per cone: qcount[c] = bits set in the cone's row.
__global__ void wl_qset_count_kernel(const uint32_t* __restrict__ B, int NC, int64_t W, uint32_t* __restrict__ qcount)
{
    const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= NC) return;
    uint32_t n = 0;
    for (int64_t w = lane; w < W; w += 32) n += __popc(B[c * W + w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) qcount[c] = n;
}

// Exclusive scan of one value per thread over a CTA of WL_CONES_THREADS
// threads; *total receives the sum.  wsum: WL_CONES_THREADS / 32 + 1 words
// (the warps' offsets, then the total).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = wsum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    const uint32_t r = wsum[warp] + incl - v;
    *total = wsum[32];
    __syncthreads();  // wsum is reused by the next scan
    return r;
}

// One CTA over all cones (N_C <= 12288): first entries (scan of the counts)
// and item offsets (scan of the item counts); item_off[N_C] = total items;
// resets the screen's work counter.
__global__ void __launch_bounds__(WL_CONES_THREADS) wl_qset_cones_kernel(const uint32_t* __restrict__ qcount, int NC,
                                                                       int G, uint32_t* __restrict__ qoff,
                                                                       uint32_t* __restrict__ item_off,
                                                                       uint32_t* __restrict__ counters)
{
    __shared__ uint32_t wsum[WL_CONES_THREADS / 32 + 1];
    const int tid = threadIdx.x;
    const int per = (NC + WL_CONES_THREADS - 1) / WL_CONES_THREADS;  // <= WL_CONES_PER
    const int c0 = tid * per < NC ? tid * per : NC, c1 = c0 + per < NC ? c0 + per : NC;
    uint32_t cnt[WL_CONES_PER], sc = 0, si = 0;
#pragma unroll
    for (int i = 0; i < WL_CONES_PER; ++i) {
        cnt[i] = c0 + i < c1 ? qcount[c0 + i] : 0u;
        sc += cnt[i];
        si += (cnt[i] + uint32_t(G) - 1) / uint32_t(G);
    }
    uint32_t tot_c, tot_i;
    uint32_t oc = block_excl_scan(sc, wsum, &tot_c);
    uint32_t oi = block_excl_scan(si, wsum, &tot_i);
#pragma unroll
    for (int i = 0; i < WL_CONES_PER; ++i)
        if (c0 + i < c1) {
            qoff[c0 + i] = oc;
            item_off[c0 + i] = oi;
            oc += cnt[i];
            oi += (cnt[i] + uint32_t(G) - 1) / uint32_t(G);
        }
    if (tid == 0) {
        item_off[NC] = tot_i;
        counters[0] = 0;  // work counter of the scan that follows
    }
}

constexpr int QSET_EXPAND_THREADS = 256;

// Warp per cone: its query set in ascending order into qlist[qoff[c] ...]
// (entry q * S), and its item descriptors.  Per 32 words of the set, each
// lane writes its word's queries into the warp's shared-memory stage at their
// ranks, then the warp copies the stage out with consecutive lanes on
// consecutive entries.
__global__ void __launch_bounds__(QSET_EXPAND_THREADS) wl_qset_expand_kernel(
    const uint32_t* __restrict__ B, int NC, int64_t W, int64_t S, const uint32_t* __restrict__ offsets,
    const uint32_t* __restrict__ qcount, const uint32_t* __restrict__ qoff, const uint32_t* __restrict__ item_off,
    int G, uint32_t* __restrict__ qlist, uint4* __restrict__ items)
{
    __shared__ uint32_t stage_all[QSET_EXPAND_THREADS / 32][32 * 32];
    const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    uint32_t* stage = stage_all[threadIdx.x >> 5];
    if (c >= NC) return;
    const uint32_t cnt = qcount[c];
    if (cnt == 0) return;
    uint32_t base = qoff[c];
    for (int64_t w0 = 0; w0 < W; w0 += 32) {
        uint32_t m = w0 + lane < W ? B[c * W + w0 + lane] : 0u;
        const uint32_t n = __popc(m);
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t pos = incl - n;
        const uint32_t qb = uint32_t(w0 + lane) * 32u;
        while (m) {
            const int j = __ffs(int(m)) - 1;
            m &= m - 1u;
            stage[pos++] = (qb + uint32_t(j)) * uint32_t(S);
        }
        __syncwarp();
        for (uint32_t r = lane; r < tot; r += 32) qlist[base + r] = stage[r];
        __syncwarp();
        base += tot;
    }
    const uint32_t o = item_off[c], ni = (cnt + uint32_t(G) - 1) / uint32_t(G);
    const uint32_t r0 = offsets[c], r1 = offsets[c + 1], q0 = qoff[c];
    for (uint32_t g = lane; g < ni; g += 32) {
        const uint32_t rest = cnt - g * uint32_t(G);
        items[o + g] = make_uint4(r0, r1, q0 + g * uint32_t(G), rest < uint32_t(G) ? rest : uint32_t(G));
    }
}

// The per-cone shared-memory arrays (N_C words and the N_C-bit non-empty
// bitmap) pass the default 48 KB of dynamic shared memory for N_C > 11904:
// raise the limit of the kernels that hold them, once per process.
static void wl_smem_attributes()
{
    static bool done[64] = {};  // per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && done[dev]) return;
    const int lim = int((12288 + 12288 / 32) * 4);
    cudaFuncSetAttribute(wl_block_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(wl_block_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(wl_qset_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaGetLastError();
    if (dev >= 0 && dev < 64) done[dev] = true;
}

int64_t wl_qset_words(int64_t NC, int64_t Q)
{
    if (NC > 12288) return 0;
    const int64_t W = (Q + 31) / 32, words = NC * W;
    return words * 4 <= (int64_t(256) << 20) ? words : 0;  // at most 256 MB of query sets
}

static int launch_worklist_qset(const uint32_t* probes, int64_t Q, int64_t S, const uint32_t* offsets, int NC, int G,
                                BatchedBuffers& b, cudaStream_t st, int num_sms)
{
    const int64_t W = (Q + 31) / 32;
    int rc;
    cudaMemsetAsync(b.qset, 0, size_t(NC) * size_t(W) * 4, st);
    const int64_t parts = (S + QSET_PCHUNK - 1) / QSET_PCHUNK;
    if (parts > 65535 || W > int64_t(0x7FFFFFFF)) return -2;  // grid limits
    const size_t sm = (size_t(NC) + size_t(NC + 31) / 32) * 4;
    wl_smem_attributes();
    wl_qset_kernel<<<dim3(unsigned(W), unsigned(parts)), QSET_THREADS, sm, st>>>(probes, Q, S, offsets, NC, W, b.qset);
    if ((rc = count_launch())) return rc;
    const unsigned wb = unsigned((int64_t(NC) * 32 + 255) / 256);
    wl_qset_count_kernel<<<wb, 256, 0, st>>>(b.qset, NC, W, b.qcount);
    if ((rc = count_launch())) return rc;
    wl_qset_cones_kernel<<<1, WL_CONES_THREADS, 0, st>>>(b.qcount, NC, G, b.qoff, b.item_off, b.counters);
    if ((rc = count_launch())) return rc;
    const unsigned eb = unsigned((int64_t(NC) * 32 + QSET_EXPAND_THREADS - 1) / QSET_EXPAND_THREADS);
    wl_qset_expand_kernel<<<eb, QSET_EXPAND_THREADS, 0, st>>>(b.qset, NC, W, S, offsets, b.qcount, b.qoff,
                                                               b.item_off, G, b.qlist, b.items);
    return count_launch();
}

int launch_worklist(const uint32_t* probes, int64_t Q, int64_t P_eff, const uint32_t* offsets, int64_t NC, int group,
                    BatchedBuffers& b, cudaStream_t st, int num_sms, bool query_only)
{
    if (query_only && b.qset && wl_qset_words(NC, Q) > 0)
        return launch_worklist_qset(probes, Q, P_eff, offsets, int(NC), group, b, st, num_sms);
    const int64_t n = Q * P_eff;
    int rc;
    int64_t cb = (NC + 256) / 256;
    if (cb > 4 * num_sms) cb = 4 * num_sms;
    if (NC <= 12288) {
        // per-block cone histograms, one scan, shared-memory cursors: no
        // contended global atomics
        const int nb = wl_blocks_impl(n, num_sms);
        const int64_t chunk = ((n + nb - 1) / nb + 3) & ~int64_t(3);  // a multiple of 4 (vector loads)
        const size_t sm = (size_t(NC) + size_t(NC + 31) / 32) * 4;     // counters + non-empty bitmap
        wl_smem_attributes();
        const int64_t hn = NC * nb + 1;
        cudaMemsetAsync(b.hbuf + NC * nb, 0, 4, st);
        wl_block_hist_kernel<<<unsigned(nb), 512, sm, st>>>(probes, n, chunk, offsets, int(NC), b.hbuf);
        if ((rc = count_launch())) return rc;
        if ((rc = launch_exclusive_scan(b.hbuf, b.hbuf, hn, b.scan_temp, st))) return rc;
        wl_cones_kernel<<<1, WL_CONES_THREADS, 0, st>>>(b.hbuf, int(NC), nb, group, b.qcount, b.qoff, b.item_off,
                                                          b.counters);
        if ((rc = count_launch())) return rc;
        wl_block_fill_kernel<<<unsigned(nb), 512, sm, st>>>(probes, n, chunk, offsets, int(NC), b.hbuf,
                                                                         b.qlist, b.qcount, b.qoff, b.item_off,
                                                                         group, b.items);
        return count_launch();
    } else {
        cudaMemsetAsync(b.qcount, 0, size_t(NC + 1) * 4, st);
        cudaMemsetAsync(b.fill, 0, size_t(NC) * 4, st);
        int64_t blocks = (n + 4095) / 4096;
        if (blocks < 1) blocks = 1;
        int64_t bl = blocks > 8 * num_sms ? 8 * num_sms : blocks;
        wl_count_global_kernel<<<unsigned(bl), 256, 0, st>>>(probes, n, offsets, uint32_t(NC), b.qcount);
        if ((rc = count_launch())) return rc;
        if ((rc = launch_exclusive_scan(b.qcount, b.qoff, NC + 1, b.scan_temp, st))) return rc;
        wl_fill_kernel<<<unsigned(bl), 256, 0, st>>>(probes, n, offsets, uint32_t(NC), b.qoff, b.fill, b.qlist);
        if ((rc = count_launch())) return rc;
    }
    wl_nitems_kernel<<<unsigned(cb), 256, 0, st>>>(b.qcount, NC, group, b.nitems);
    if ((rc = count_launch())) return rc;
    if ((rc = launch_exclusive_scan(b.nitems, b.item_off, NC + 1, b.scan_temp, st))) return rc;
    wl_items_kernel<<<unsigned(cb), 256, 0, st>>>(b.nitems, b.item_off, offsets, b.qcount, b.qoff, NC, group,
                                                   b.items, b.counters);
    if ((rc = count_launch())) return rc;
    return 0;
}

// ---------------------------------------------------------------- tile scan

struct TileArgs {
    const float* xs;           // rows, stride d_pad
    const uint32_t* offsets;   // cone offsets (sparse mode)
    const uint32_t* perm;      // row -> point id
    const float* Y;            // queries, stride d
    const int64_t* query_src;  // exclusion sources (nullable)
    const uint4* items;        // sparse mode: (first row, end row, first slot, slot count)
    const uint32_t* n_items_dev;
    const uint32_t* qcount;
    const uint32_t* qoff;
    const uint32_t* qlist;     // slot ids = q * S + s
    uint32_t* counter;
    uint64_t* partial;         // [Q * S * k]
    uint32_t* status;
    int64_t S;                 // slots per query
    int64_t grid_w;
    int64_t N, Q;              // dense mode sizes
    int64_t n_groups, n_items_dense;
    int d_pad, d, k, radius;
    int dense;                 // 1: linear search items
};

struct ItemDesc {
    uint32_t row0, row1;  // rows of the item
    uint32_t qbeg, qn;    // slot list range (sparse) or first query and count (dense)
    uint32_t chunk;       // dense: chunk index = slot offset
};

__device__ __forceinline__ ItemDesc load_item(const TileArgs& a, uint32_t item, int G)
{
    ItemDesc it;
    if (a.dense) {
        const uint32_t c = item / uint32_t(a.n_groups), g = item % uint32_t(a.n_groups);
        it.row0 = c * BF_CHUNK_ROWS;
        const int64_t e = int64_t(it.row0) + BF_CHUNK_ROWS;
        it.row1 = uint32_t(e < a.N ? e : a.N);
        it.qbeg = g * uint32_t(G);
        const int64_t qe = int64_t(it.qbeg) + G;
        it.qn = uint32_t((qe < a.Q ? qe : a.Q) - it.qbeg);
        it.chunk = c;
    } else {
        const uint4 d = a.items[item];
        it.row0 = d.x;
        it.row1 = d.y;
        it.qbeg = d.z;
        it.qn = d.w;
        it.chunk = 0;
    }
    return it;
}

template <int DPT, int KMAX, bool EXCL>
__global__ void __launch_bounds__(TILE_THREADS) tile_scan_kernel(const TileArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage_buf = reinterpret_cast<float*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[TILE_STAGES];
    __shared__ int4 meta[TILE_STAGES];  // (first row, rows or -1, item, last chunk of item)
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int TPR = a.d_pad / DPT;
    const int G = TILE_THREADS / TPR;
    const int RPC = TILE_STAGE_FLOATS / a.d_pad;
    const int qs = tid / TPR, sub = tid % TPR;
    const uint32_t n_items = a.dense ? uint32_t(a.n_items_dense) : *a.n_items_dev;

    // producer state (thread 0 only)
    bool done = false;
    int cur_item = -1;
    uint32_t cur = 0, cur_end = 0;
    auto issue = [&](int s) {
        while (!done && cur >= cur_end) {
            const uint32_t it = atomicAdd(a.counter, 1u);
            if (it >= n_items) {
                done = true;
                break;
            }
            const ItemDesc d = load_item(a, it, G);
            cur_item = int(it);
            cur = d.row0;
            cur_end = d.row1;
        }
        if (done) {
            meta[s] = make_int4(0, -1, -1, 0);
            return;
        }
        const uint32_t n = cur_end - cur < uint32_t(RPC) ? cur_end - cur : uint32_t(RPC);
        meta[s] = make_int4(int(cur), int(n), cur_item, cur + n == cur_end ? 1 : 0);
        const uint32_t bytes = n * uint32_t(a.d_pad) * 4u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(stage_buf + size_t(s) * TILE_STAGE_FLOATS, a.xs + size_t(cur) * a.d_pad, bytes, &bars[s]);
        cur += n;
    };

    if (tid == 0) {
        for (int s = 0; s < TILE_STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < TILE_STAGES; ++s) issue(s);
    __syncthreads();

    float4 qv[DPT / 4];
    uint64_t list[KMAX];
    int item = -1;
    bool active = false;
    int64_t slot = 0, src = -1;

    int c = 0;
    for (;; ++c) {
        const int s = c % TILE_STAGES;
        const int4 m = meta[s];
        if (m.y < 0) break;
        if (m.z != item) {
            // first chunk of a new item: load this thread's query slice
            item = m.z;
            const ItemDesc d = load_item(a, uint32_t(item), G);
            active = uint32_t(qs) < d.qn;
            int64_t q = 0;
            if (active) {
                if (a.dense) {
                    q = int64_t(d.qbeg) + qs;
                    slot = q * a.S + d.chunk;
                } else {
                    slot = int64_t(a.qlist[d.qbeg + qs]);
                    q = slot / a.S;
                }
            }
            const float* y = a.Y + q * int64_t(a.d);
#pragma unroll
            for (int jj = 0; jj < DPT / 4; ++jj) {
                const int cc = sub * DPT + jj * 4;
                qv[jj].x = active && cc + 0 < a.d ? y[cc + 0] : 0.0f;
                qv[jj].y = active && cc + 1 < a.d ? y[cc + 1] : 0.0f;
                qv[jj].z = active && cc + 2 < a.d ? y[cc + 2] : 0.0f;
                qv[jj].w = active && cc + 3 < a.d ? y[cc + 3] : 0.0f;
            }
            if (EXCL) src = active ? a.query_src[q] : -1;
            topk_init<KMAX>(list, a.k);
        }
        const bool ok = mbar_wait_bounded(&bars[s], uint32_t((c / TILE_STAGES) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.status, ST_TIMEOUT);
                abort_flag = 1;
            }
            break;
        }
        const float* base = stage_buf + size_t(s) * TILE_STAGE_FLOATS + sub * DPT;
        const int n = m.y;
        for (int r = 0; r < n; r += 4) {
            // canonical piece tree (osann_device.cuh), four rows at a time;
            // rows past the chunk read stale stage memory and are discarded
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4* row = reinterpret_cast<const float4*>(base + (r + u) * a.d_pad);
                float cpart[DPT / 4];
#pragma unroll
                for (int jj = 0; jj < DPT / 4; ++jj) cpart[jj] = sq4(row[jj], qv[jj]);
                acc[u] = pair_tree<DPT / 4>(cpart);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = lane_tree(acc[u], TPR);
            if (active && sub == 0) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (r + u < n) {
                        const uint32_t row = uint32_t(m.x + r + u);
                        if (EXCL) {
                            const uint32_t id = a.perm ? __ldg(a.perm + row) : row;
                            const int64_t dr = int64_t(id) / a.grid_w - src / a.grid_w;
                            const int64_t dc = int64_t(id) % a.grid_w - src % a.grid_w;
                            const int64_t ch = (dr < 0 ? -dr : dr) > (dc < 0 ? -dc : dc) ? (dr < 0 ? -dr : dr)
                                                                                          : (dc < 0 ? -dc : dc);
                            if (src < 0 || ch > a.radius) {
                                const uint64_t v = pack_di(acc[u], id);
                                if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                            }
                        } else if (acc[u] <= di_dist(list[KMAX - 1])) {
                            const uint32_t id = a.perm ? __ldg(a.perm + row) : row;
                            const uint64_t v = pack_di(acc[u], id);
                            if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                        }
                    }
                }
            }
        }
        if (m.w && active && sub == 0) {
            uint64_t* out = a.partial + slot * a.k;
#pragma unroll
            for (int j = 0; j < KMAX; ++j)
                if (j >= KMAX - a.k) out[j - (KMAX - a.k)] = list[j];
        }
        __syncthreads();
        if (tid == 0) issue(s);
    }
    if (abort_flag) {
        if (tid == 0)
            for (int i = 0; i < TILE_STAGES; ++i) {
                const int cc = c + i, ss = cc % TILE_STAGES;
                if (meta[ss].y >= 0) mbar_wait_bounded(&bars[ss], uint32_t((cc / TILE_STAGES) & 1));
            }
        __syncthreads();
    }
}

template <int DPT, int KMAX, bool EXCL>
static int launch_tile_t(const TileArgs& a, cudaStream_t st, int num_sms)
{
    const int smem = TILE_STAGES * TILE_STAGE_FLOATS * 4;
    auto kern = tile_scan_kernel<DPT, KMAX, EXCL>;
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TILE_THREADS, smem);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    kern<<<unsigned(num_sms * blocks_per_sm), TILE_THREADS, smem, st>>>(a);
    return count_launch();
}

template <int DPT, bool EXCL>
static int launch_tile_k(const TileArgs& a, cudaStream_t st, int num_sms)
{
    if (a.k <= 1) return launch_tile_t<DPT, 1, EXCL>(a, st, num_sms);
    if (a.k <= 4) return launch_tile_t<DPT, 4, EXCL>(a, st, num_sms);
    if (a.k <= 16) return launch_tile_t<DPT, 16, EXCL>(a, st, num_sms);
    return launch_tile_t<DPT, 32, EXCL>(a, st, num_sms);
}

static int launch_tile_any(const TileArgs& a, cudaStream_t st, int num_sms)
{
    const bool excl = a.query_src != nullptr;
    if (a.d_pad == 16) return excl ? launch_tile_k<16, true>(a, st, num_sms) : launch_tile_k<16, false>(a, st, num_sms);
    return excl ? launch_tile_k<32, true>(a, st, num_sms) : launch_tile_k<32, false>(a, st, num_sms);
}

int launch_tile_scan(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad, const float* Y, int d,
                     int64_t slots_per_query, int k, const int64_t* query_src, int64_t grid_w, int radius,
                     const BatchedBuffers& b, int group, uint64_t* partial, uint32_t* status, cudaStream_t st,
                     int num_sms)
{
    (void)group;
    TileArgs a{};
    a.xs = xs;
    a.offsets = offsets;
    a.perm = perm;
    a.Y = Y;
    a.query_src = query_src;
    a.items = b.items;
    a.n_items_dev = b.n_items_dev;
    a.qcount = b.qcount;
    a.qoff = b.qoff;
    a.qlist = b.qlist;
    a.counter = b.counters;
    a.partial = partial;
    a.status = status;
    a.S = slots_per_query;
    a.grid_w = grid_w;
    a.d_pad = d_pad;
    a.d = d;
    a.k = k;
    a.radius = radius;
    a.dense = 0;
    return launch_tile_any(a, st, num_sms);
}

// ---------------------------------------------------------------- merge

template <int KMAX>
__global__ void __launch_bounds__(128) merge_kernel(const uint64_t* __restrict__ partial, int64_t Q, int64_t S, int k,
                                                    int64_t* __restrict__ out_ids, float* __restrict__ out_d)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const uint64_t* p = partial + q * S * k;
    const int64_t n = S * k;
    // each lane keeps the k best of its share, then k rounds of warp minimum
    uint64_t list[KMAX];
    topk_init<KMAX>(list, k);
    for (int64_t i = lane; i < n; i += 32) {
        const uint64_t v = p[i];
        if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
    }
    for (int j = 0; j < k; ++j) {
        const uint64_t head = topk_head<KMAX>(list, k);
        const uint64_t best = warp_min_u64(head);
        if (head == best && best != EMPTY_DI) topk_remove<KMAX>(list, k, best);
        if (lane == 0) {
            const uint32_t id = di_id(best);
            out_ids[q * k + j] = id == 0xFFFFFFFFu ? int64_t(-1) : int64_t(id);
            out_d[q * k + j] = di_dist(best);
        }
    }
}

int launch_merge(const uint64_t* partial, int64_t Q, int64_t S, int k, const uint32_t* perm_or_null, int64_t* out_ids,
                 float* out_d, cudaStream_t st)
{
    (void)perm_or_null;
    if (Q == 0) return 0;
    const unsigned blocks = unsigned((Q * 32 + 127) / 128);
    if (k <= 1) merge_kernel<1><<<blocks, 128, 0, st>>>(partial, Q, S, k, out_ids, out_d);
    else if (k <= 4) merge_kernel<4><<<blocks, 128, 0, st>>>(partial, Q, S, k, out_ids, out_d);
    else if (k <= 16) merge_kernel<16><<<blocks, 128, 0, st>>>(partial, Q, S, k, out_ids, out_d);
    else merge_kernel<32><<<blocks, 128, 0, st>>>(partial, Q, S, k, out_ids, out_d);
    return count_launch();
}

// ---------------------------------------------------------------- linear search

size_t bruteforce_ws_bytes(int64_t N, int d_pad, int64_t Q, int k)
{
    const int64_t S = (N + BF_CHUNK_ROWS - 1) / BF_CHUNK_ROWS;
    (void)d_pad;
    return size_t(Q) * size_t(S) * size_t(k) * 8 + 256;
}

__global__ void fill_u64_kernel(uint64_t* __restrict__ p, int64_t n, uint64_t v)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = v;
}

int launch_bruteforce_rows(const float* xs, const uint32_t* perm, int64_t N, int d_pad, const float* Y, int d,
                           int64_t Q, int k, const int64_t* query_src, int64_t grid_w, int radius, void* ws,
                           uint32_t* counter, int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st,
                           int num_sms)
{
    if (Q == 0) return 0;
    const int64_t S = (N + BF_CHUNK_ROWS - 1) / BF_CHUNK_ROWS;
    uint64_t* partial = static_cast<uint64_t*>(ws);
    const int64_t np = Q * S * k;
    int64_t fb = (np + 255) / 256;
    if (fb > 8 * num_sms) fb = 8 * num_sms;
    if (fb < 1) fb = 1;
    fill_u64_kernel<<<unsigned(fb), 256, 0, st>>>(partial, np, EMPTY_DI);
    int rc = count_launch();
    if (rc) return rc;
    if (N > 0) {
        const int DPT = d_pad == 16 ? 16 : 32;
        const int G = TILE_THREADS / (d_pad / DPT);
        cudaMemsetAsync(counter, 0, 4, st);
        TileArgs a{};
        a.xs = xs;
        a.perm = perm;
        a.Y = Y;
        a.query_src = query_src;
        a.counter = counter;
        a.partial = partial;
        a.status = status;
        a.S = S;
        a.grid_w = grid_w;
        a.N = N;
        a.Q = Q;
        a.n_groups = (Q + G - 1) / G;
        a.n_items_dense = S * a.n_groups;
        a.d_pad = d_pad;
        a.d = d;
        a.k = k;
        a.radius = radius;
        a.dense = 1;
        if ((rc = launch_tile_any(a, st, num_sms))) return rc;
    }
    return launch_merge(partial, Q, S, k, nullptr, out_ids, out_d, st);
}

}  // namespace osann
