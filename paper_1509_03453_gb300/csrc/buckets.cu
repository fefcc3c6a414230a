// Bucket index build: cone histogram, exclusive scan (CSR offsets), stable
// counting sort of point ids by cone, and the gather of the permuted vectors.
//
// The paper keeps one hash table per basis mapping each cone to its points
// (Sec. 4, preparation phase).  Here the table is a CSR layout:
//   offsets[N_C + 1]  exclusive prefix sum of the cone counts,
//   perm[N]           point ids, ascending inside every cone (stable order),
//   xs[N x d_pad]     the vectors in perm order, fp32, zero padded,
//   rowstat[N]        ((1-B)|x|^2, |x|, |x|^2, 0) for the tensor-core screen,
//   x16, xe16         (optional) the screen's fp16 operands, written here so
//                     the vectors are read once.
// Nothing here spins on another block: the scan is reduce-then-scan, the sort
// is a least-significant-digit radix sort whose passes are stable by lane
// rank inside each warp chunk and by chunk order across chunks.
#include "osann_device.cuh"
#include "osann_launch.h"

#include <cuda_fp16.h>

namespace osann {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------- scan

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = s;
    }
    __syncthreads();
    return x - v + warp_sums[warp];
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                   uint32_t* __restrict__ sums)
{
    __shared__ uint32_t ws[32];
    const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i * SCAN_THREADS + threadIdx.x;
        if (j < n) s += in[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of one tile per block, plus the block's offset (if any).
// Safe in place: the whole tile is read before any of it is written.
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_kernel(const uint32_t* in, uint32_t* out, int64_t n,
                                                                 const uint32_t* __restrict__ block_off)
{
    __shared__ uint32_t tile[SCAN_TILE];
    __shared__ uint32_t ws[32];
    __shared__ uint32_t total;
    const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i * SCAN_THREADS + threadIdx.x;
        tile[i * SCAN_THREADS + threadIdx.x] = j < n ? in[j] : 0u;
    }
    __syncthreads();
    uint32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = tile[threadIdx.x * SCAN_ITEMS + i];
        s += v[i];
    }
    uint32_t pre = block_exclusive_scan(s, ws, &total);
    if (block_off) pre += block_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        tile[threadIdx.x * SCAN_ITEMS + i] = pre;
        pre += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i * SCAN_THREADS + threadIdx.x;
        if (j < n) out[j] = tile[i * SCAN_THREADS + threadIdx.x];
    }
}

size_t scan_temp_bytes(int64_t n)
{
    size_t b = 0;
    while (n > SCAN_TILE) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        b += size_t((n + 63) / 64 * 64) * sizeof(uint32_t);
    }
    return b + 256;
}

int launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t st)
{
    if (n <= 0) return 0;
    if (n <= SCAN_TILE) {
        scan_tile_kernel<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr);
        return count_launch();
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* sums = static_cast<uint32_t*>(temp);
    void* rest = sums + (nb + 63) / 64 * 64;
    scan_reduce_kernel<<<unsigned(nb), SCAN_THREADS, 0, st>>>(in, n, sums);
    int rc = count_launch();
    if (rc) return rc;
    rc = launch_exclusive_scan(sums, sums, nb, rest, st);
    if (rc) return rc;
    scan_tile_kernel<<<unsigned(nb), SCAN_THREADS, 0, st>>>(in, out, n, sums);
    return count_launch();
}

// ---------------------------------------------------------------- histogram

__global__ void __launch_bounds__(512) hist_smem_kernel(const uint32_t* __restrict__ keys, int64_t N, int NC,
                                                        uint32_t* __restrict__ counts)
{
    extern __shared__ uint32_t h[];
    for (int c = threadIdx.x; c < NC; c += blockDim.x) h[c] = 0;
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    {
        const uint32_t key = keys[i];
        if (key < uint32_t(NC)) atomicAdd(&h[key], 1u);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NC; c += blockDim.x)
        if (h[c]) atomicAdd(&counts[c], h[c]);
}

__global__ void hist_global_kernel(const uint32_t* __restrict__ keys, int64_t N, int64_t NC,
                                   uint32_t* __restrict__ counts)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t key = keys[i];
        if (key < NC) atomicAdd(&counts[key], 1u);
    }
}

int launch_key_histogram(const uint32_t* keys, int64_t N, int64_t NC, uint32_t* counts, cudaStream_t st,
                         int num_sms)
{
    if (N == 0) return 0;
    int64_t blocks = (N + 4095) / 4096;
    if (NC <= 12288) {
        if (blocks > 2 * num_sms) blocks = 2 * num_sms;
        hist_smem_kernel<<<unsigned(blocks), 512, size_t(NC) * 4, st>>>(keys, N, int(NC), counts);
    } else {
        if (blocks > 8 * num_sms) blocks = 8 * num_sms;
        hist_global_kernel<<<unsigned(blocks), 256, 0, st>>>(keys, N, NC, counts);
    }
    return count_launch();
}

// ---------------------------------------------------------------- radix sort

constexpr int RADIX_CHUNK = 2048;  // elements per chunk (one CTA)
constexpr int RADIX_WARPS = 8;     // warps per CTA, RADIX_CHUNK / RADIX_WARPS elements each
constexpr int RADIX_WE = RADIX_CHUNK / RADIX_WARPS;

struct RadixPlan {
    int passes, bits_per_pass, B;
    int64_t nchunks;
};

static RadixPlan radix_plan_bits(int64_t N, int bits)
{
    RadixPlan p;
    p.passes = (bits + 10) / 11;
    p.bits_per_pass = (bits + p.passes - 1) / p.passes;
    p.B = 1 << p.bits_per_pass;
    p.nchunks = (N + RADIX_CHUNK - 1) / RADIX_CHUNK;
    return p;
}

static RadixPlan radix_plan(int64_t N, int64_t NC)
{
    int bits = 1;
    while ((int64_t(1) << bits) < NC) ++bits;
    return radix_plan_bits(N, bits);
}

// Digit of element i: bits [shift, shift + log2 B) of its key.  WIDE: the key
// is the 128-bit id of the element's point (ids_in[i], or i in the first
// pass), read from wkeys, instead of a carried 32-bit key.
template <bool WIDE>
__device__ __forceinline__ uint32_t radix_digit(const uint32_t* __restrict__ keys, const uint4* __restrict__ wkeys,
                                                const uint32_t* __restrict__ ids_in, int64_t i, int shift,
                                                uint32_t mask)
{
    if (WIDE) {
        const uint32_t id = ids_in ? ids_in[i] : uint32_t(i);
        return uint32_t(wide_value(wkeys[id]) >> shift) & mask;
    }
    return (keys[i] >> shift) & mask;
}

// Digit counts of one chunk: H[digit * nchunks + chunk].
template <bool WIDE>
__global__ void __launch_bounds__(RADIX_WARPS * 32) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                      const uint4* __restrict__ wkeys,
                                                                      const uint32_t* __restrict__ ids_in, int64_t N,
                                                                      int shift, int B, int64_t nchunks,
                                                                      uint32_t* __restrict__ H)
{
    extern __shared__ uint32_t sh[];
    const int64_t chunk = blockIdx.x;
    for (int i = threadIdx.x; i < B; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t begin = chunk * RADIX_CHUNK;
    const int64_t end = begin + RADIX_CHUNK < N ? begin + RADIX_CHUNK : N;
    const uint32_t mask = uint32_t(B - 1);
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&sh[radix_digit<WIDE>(keys, wkeys, ids_in, i, shift, mask)], 1u);
    __syncthreads();
    for (int dg = threadIdx.x; dg < B; dg += blockDim.x) H[int64_t(dg) * nchunks + chunk] = sh[dg];
}

// Stable scatter of one chunk.  Warp w owns elements [w * RADIX_WE, (w + 1) *
// RADIX_WE) of the chunk: (1) per-warp digit counts in shared memory, (2) for
// each digit a running sum over the warps from the chunk's scanned base, (3)
// each warp places its elements in order (match_any ranks within a round).
template <bool WIDE>
__global__ void __launch_bounds__(RADIX_WARPS * 32) radix_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint4* __restrict__ wkeys, const uint32_t* __restrict__ ids_in,
    int64_t N, int shift, int B,
    int64_t nchunks, const uint32_t* __restrict__ Hs, uint32_t* __restrict__ keys_out, uint32_t* __restrict__ ids_out,
    uint32_t* __restrict__ offsets_out, int64_t NC)
{
    extern __shared__ uint32_t sh[];  // [RADIX_WARPS][B]
    // single pass over all key bits: the scanned counts at chunk 0 are the
    // bucket starts (CSR offsets)
    if (offsets_out && blockIdx.x == 0)
        for (int64_t dg = threadIdx.x; dg <= NC; dg += blockDim.x)
            offsets_out[dg] = dg < NC ? Hs[dg * nchunks] : uint32_t(N);
    constexpr int R = RADIX_WE / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = blockIdx.x;
    const int64_t wbeg = chunk * RADIX_CHUNK + int64_t(warp) * RADIX_WE;
    const int64_t wend = wbeg + RADIX_WE < N ? wbeg + RADIX_WE : N;
    const uint32_t mask = uint32_t(B - 1);
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < RADIX_WARPS * B; i += blockDim.x) sh[i] = 0;
    uint32_t key[R], id[R], digit[R];
    unsigned peers[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = wbeg + 32 * r + lane;
        const bool live = i < wend;
        key[r] = live && !WIDE ? keys_in[i] : 0u;
        id[r] = live ? (ids_in ? ids_in[i] : uint32_t(i)) : 0u;
        digit[r] = !live ? 0xFFFFFFFFu
                         : (WIDE ? radix_digit<true>(keys_in, wkeys, ids_in, i, shift, mask) : (key[r] >> shift) & mask);
    }
    __syncthreads();
    uint32_t* cnt = sh + warp * B;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        peers[r] = __match_any_sync(0xffffffffu, digit[r]);
        if (digit[r] != 0xFFFFFFFFu && lane == __ffs(peers[r]) - 1) cnt[digit[r]] += __popc(peers[r]);
        __syncwarp();
    }
    __syncthreads();
    for (int dg = threadIdx.x; dg < B; dg += blockDim.x) {
        uint32_t run = Hs[int64_t(dg) * nchunks + chunk];
#pragma unroll
        for (int w = 0; w < RADIX_WARPS; ++w) {
            const uint32_t c = sh[w * B + dg];
            sh[w * B + dg] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool live = digit[r] != 0xFFFFFFFFu;
        if (live) {
            const uint32_t pos = cnt[digit[r]] + __popc(peers[r] & lt);
            ids_out[pos] = id[r];
            if (!WIDE && keys_out) keys_out[pos] = key[r];
        }
        __syncwarp();
        if (live && lane == __ffs(peers[r]) - 1) cnt[digit[r]] += __popc(peers[r]);
        __syncwarp();
    }
}

size_t radix_temp_bytes(int64_t N, int64_t NC)
{
    RadixPlan p = radix_plan(N, NC);
    const int64_t hn = int64_t(p.B) * p.nchunks;
    size_t b = size_t((hn + 63) / 64 * 64) * 4;
    b += scan_temp_bytes(hn);
    b += size_t((N + 63) / 64 * 64) * 4 * 4;  // two (keys, ids) ping-pong pairs
    return b + 1024;
}

bool radix_single_pass(int64_t NC) { return radix_plan(1, NC).passes == 1; }

int launch_stable_sort_ids(const uint32_t* keys, int64_t N, int64_t NC, uint32_t* perm, uint32_t* offsets, void* temp,
                           cudaStream_t st)
{
    if (N == 0) {
        if (offsets && cudaMemsetAsync(offsets, 0, size_t(NC + 1) * 4, st) != cudaSuccess) return -5;
        return 0;
    }
    RadixPlan p = radix_plan(N, NC);
    const int64_t hn = int64_t(p.B) * p.nchunks;
    char* t = static_cast<char*>(temp);
    uint32_t* H = reinterpret_cast<uint32_t*>(t);
    t += size_t((hn + 63) / 64 * 64) * 4;
    void* stemp = t;
    t += (scan_temp_bytes(hn) + 255) / 256 * 256;
    const size_t nb = size_t((N + 63) / 64 * 64) * 4;
    uint32_t* ka = reinterpret_cast<uint32_t*>(t);
    uint32_t* ia = reinterpret_cast<uint32_t*>(t + nb);
    uint32_t* kb = reinterpret_cast<uint32_t*>(t + 2 * nb);
    uint32_t* ib = reinterpret_cast<uint32_t*>(t + 3 * nb);
    const unsigned blocks = unsigned(p.nchunks);
    const size_t hsmem = size_t(p.B) * 4, smem = size_t(RADIX_WARPS) * p.B * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(radix_scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(RADIX_WARPS * 2048 * 4));
        attr_set = true;
    }
    const uint32_t* kin = keys;
    const uint32_t* iin = nullptr;
    for (int pass = 0; pass < p.passes; ++pass) {
        const int shift = pass * p.bits_per_pass;
        const bool last = pass == p.passes - 1;
        uint32_t* kout = last ? nullptr : (pass % 2 == 0 ? ka : kb);
        uint32_t* iout = last ? perm : (pass % 2 == 0 ? ia : ib);
        radix_hist_kernel<false><<<blocks, RADIX_WARPS * 32, hsmem, st>>>(kin, nullptr, nullptr, N, shift, p.B,
                                                                         p.nchunks, H);
        int rc = count_launch();
        if (rc) return rc;
        rc = launch_exclusive_scan(H, H, hn, stemp, st);
        if (rc) return rc;
        radix_scatter_kernel<false><<<blocks, RADIX_WARPS * 32, smem, st>>>(kin, nullptr, iin, N, shift, p.B,
                                                                            p.nchunks, H, kout, iout,
                                                                            p.passes == 1 ? offsets : nullptr, NC);
        rc = count_launch();
        if (rc) return rc;
        kin = kout;
        iin = iout;
    }
    return 0;
}

size_t radix_temp_bytes_wide(int64_t N, int key_bits)
{
    RadixPlan p = radix_plan_bits(N, key_bits < 1 ? 1 : key_bits);
    const int64_t hn = int64_t(p.B) * p.nchunks;
    size_t b = size_t((hn + 63) / 64 * 64) * 4;
    b += (scan_temp_bytes(hn) + 255) / 256 * 256;
    b += size_t((N + 63) / 64 * 64) * 4 * 2;  // ids ping-pong
    return b + 1024;
}

// Passes over the key_bits significant bits of the 128-bit ids, at most 11
// bits each; ids are carried, keys read through them.
int launch_stable_sort_wide(const uint4* wkeys, int64_t N, int key_bits, uint32_t* perm, void* temp, cudaStream_t st)
{
    if (N == 0) return 0;
    RadixPlan p = radix_plan_bits(N, key_bits < 1 ? 1 : key_bits);
    const int64_t hn = int64_t(p.B) * p.nchunks;
    char* t = static_cast<char*>(temp);
    uint32_t* H = reinterpret_cast<uint32_t*>(t);
    t += size_t((hn + 63) / 64 * 64) * 4;
    void* stemp = t;
    t += (scan_temp_bytes(hn) + 255) / 256 * 256;
    const size_t nb = size_t((N + 63) / 64 * 64) * 4;
    uint32_t* ia = reinterpret_cast<uint32_t*>(t);
    uint32_t* ib = reinterpret_cast<uint32_t*>(t + nb);
    const unsigned blocks = unsigned(p.nchunks);
    const size_t hsmem = size_t(p.B) * 4, smem = size_t(RADIX_WARPS) * p.B * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(radix_scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(RADIX_WARPS * 2048 * 4));
        attr_set = true;
    }
    const uint32_t* iin = nullptr;
    for (int pass = 0; pass < p.passes; ++pass) {
        const int shift = pass * p.bits_per_pass;
        uint32_t* iout = pass == p.passes - 1 ? perm : (pass % 2 == 0 ? ia : ib);
        radix_hist_kernel<true><<<blocks, RADIX_WARPS * 32, hsmem, st>>>(nullptr, wkeys, iin, N, shift, p.B,
                                                                        p.nchunks, H);
        int rc = count_launch();
        if (rc) return rc;
        rc = launch_exclusive_scan(H, H, hn, stemp, st);
        if (rc) return rc;
        radix_scatter_kernel<true><<<blocks, RADIX_WARPS * 32, smem, st>>>(nullptr, wkeys, iin, N, shift, p.B,
                                                                           p.nchunks, H, nullptr, iout, nullptr, 0);
        rc = count_launch();
        if (rc) return rc;
        iin = iout;
    }
    return 0;
}

// ---------------------------------------------------------------- gather

// One group of LPV lanes per output row; lane l owns float4 slots l, l+LPV
// of the padded row.  VEC: source rows are 16-byte aligned (d % 4 == 0).
template <int LPV, bool VEC>
__global__ void __launch_bounds__(256) gather_rows_kernel(const float* __restrict__ X, int64_t N, int d, int d_pad,
                                                         const uint32_t* __restrict__ perm, float* __restrict__ xs,
                                                         float4* __restrict__ rowstat, float Bn,
                                                         const float* __restrict__ tcs, uint16_t* __restrict__ x16,
                                                         uint16_t* __restrict__ xe16)
{
    const float sc = tcs ? tcs[0] : 1.0f, sc2 = tcs ? tcs[1] : 1.0f;
    const int lane = threadIdx.x & 31;
    const int glane = lane & (LPV - 1);
    const int64_t gid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / LPV;
    const int64_t ngroups = int64_t(gridDim.x) * blockDim.x / LPV;
    const int64_t iters = (N + ngroups - 1) / ngroups;
    const int n4p = d_pad >> 2;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t r = gid + it * ngroups;
        const bool live = r < N;
        const int64_t src = live ? int64_t(__ldg(perm + r)) : 0;
        const float* xr = X + src * int64_t(d);
        float s = 0.0f;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const int i4 = glane + f * LPV;
            if (live && i4 < n4p) {
                float4 v;
                if (VEC) {
                    v = (4 * i4 < d) ? __ldg(reinterpret_cast<const float4*>(xr) + i4) : make_float4(0, 0, 0, 0);
                } else {
                    const int c = 4 * i4;
                    v.x = c + 0 < d ? __ldg(xr + c + 0) : 0.0f;
                    v.y = c + 1 < d ? __ldg(xr + c + 1) : 0.0f;
                    v.z = c + 2 < d ? __ldg(xr + c + 2) : 0.0f;
                    v.w = c + 3 < d ? __ldg(xr + c + 3) : 0.0f;
                }
                reinterpret_cast<float4*>(xs + r * int64_t(d_pad))[i4] = v;
                if (x16) {
                    // fp16 operands of the tensor-core screen: s x, s a power of two
                    const __half2 lo = __floats2half2_rn(sc * v.x, sc * v.y), hi = __floats2half2_rn(sc * v.z, sc * v.w);
                    uint2 pk;
                    pk.x = *reinterpret_cast<const uint32_t*>(&lo);
                    pk.y = *reinterpret_cast<const uint32_t*>(&hi);
                    reinterpret_cast<uint2*>(x16 + r * int64_t(d_pad))[i4] = pk;
                }
                s = fmaf(v.x, v.x, s);
                s = fmaf(v.y, v.y, s);
                s = fmaf(v.z, v.z, s);
                s = fmaf(v.w, v.w, s);
            }
        }
#pragma unroll
        for (int m = LPV / 2; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (live && glane == 0) {
            rowstat[r] = make_float4(s * (1.0f - Bn), sqrtf(s), s, 0.0f);
            if (xe16) {
                // extra K block: fp16 hi/lo of (1-B) s^2 |x|^2 and s |x|, then zeros
                const float a = sc2 * s * (1.0f - Bn), b = sc * sqrtf(s);
                const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
                const __half al = __float2half_rn(a - __half2float(ah)), bl = __float2half_rn(b - __half2float(bh));
                uint4* dst = reinterpret_cast<uint4*>(xe16 + r * 16);
                dst[0] = make_uint4(uint32_t(__half_as_ushort(ah)) | (uint32_t(__half_as_ushort(al)) << 16),
                                    uint32_t(__half_as_ushort(bh)) | (uint32_t(__half_as_ushort(bl)) << 16), 0u, 0u);
                dst[1] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

int launch_gather_rows(const float* X, int64_t N, int d, int d_pad, const uint32_t* perm, float* xs, float4* rowstat,
                       float Bn, const float* tcs, uint16_t* x16, uint16_t* xe16, cudaStream_t st, int num_sms)
{
    if (N == 0) return 0;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const int n4p = d_pad / 4;
    int lpv = 4;
    while (lpv < n4p && lpv < 32) lpv <<= 1;
    int64_t blocks = (N * lpv + 255) / 256;
    if (blocks > int64_t(num_sms) * 16) blocks = int64_t(num_sms) * 16;
    const dim3 g(static_cast<unsigned>(blocks)), b(256u);
#define OSANN_GATHER(LP)                                                                                 \
    if (vec)                                                                                             \
        gather_rows_kernel<LP, true><<<g, b, 0, st>>>(X, N, d, d_pad, perm, xs, rowstat, Bn, tcs, x16, xe16); \
    else                                                                                                 \
        gather_rows_kernel<LP, false><<<g, b, 0, st>>>(X, N, d, d_pad, perm, xs, rowstat, Bn, tcs, x16, xe16);
    switch (lpv) {
    case 4: OSANN_GATHER(4); break;
    case 8: OSANN_GATHER(8); break;
    case 16: OSANN_GATHER(16); break;
    default: OSANN_GATHER(32); break;
    }
#undef OSANN_GATHER
    return count_launch();
}

__global__ void max_bucket_kernel(const uint32_t* __restrict__ offsets, int64_t NC, uint32_t* __restrict__ out,
                                  uint32_t* __restrict__ occ)
{
    uint32_t m = 0, n = 0;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < NC; c += int64_t(gridDim.x) * blockDim.x) {
        uint32_t s = offsets[c + 1] - offsets[c];
        m = s > m ? s : m;
        n += s > 0 ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
    if ((threadIdx.x & 31) == 0 && occ && n) atomicAdd(occ, n);
}

int launch_max_bucket(const uint32_t* offsets, int64_t NC, uint32_t* out_max, cudaStream_t st, uint32_t* out_occ)
{
    int64_t blocks = (NC + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    max_bucket_kernel<<<unsigned(blocks), 256, 0, st>>>(offsets, NC, out_max, out_occ);
    return count_launch();
}

}  // namespace osann
