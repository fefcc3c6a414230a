// Device-side helpers shared by the osann CUDA kernels (sm_103a).
//
// Packed (distance, id) keys, warp reductions, and thin inline-PTX wrappers
// for mbarriers and the bulk-copy (TMA) engine.  Every spin-wait here is
// bounded: it gives up after a clock budget and reports failure to the
// caller, which records OSANN_ST_TIMEOUT in the device status word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace osann {

// Device status word bits (OR-ed in by kernels, read by the host).
enum : uint32_t {
    ST_NONFINITE_DATA = 1u,
    ST_NONFINITE_QUERY = 2u,
    ST_TIMEOUT = 4u,
    ST_OVERFLOW = 8u,
    ST_BOUND = 16u,  // a debug check of the screening error bound failed
};

constexpr int MAX_D = 256;
constexpr int MAX_L = 16;
constexpr int MAX_K = 32;

// ---------------------------------------------------------------- wide cone ids
// When N_C reaches 2^31 (the second-level table of Sec. 4) a cone id is the
// same number rank(S) * 2^L + sign code, held in 128 bits (N_C < 2^127 for
// every d <= MAX_D, L <= MAX_L) and stored as four 32-bit words, low first.
typedef unsigned __int128 u128;

// C(n, k) in 128 bits from a table of (low, high) words, n <= MAX_D, k <= MAX_L.
__device__ __forceinline__ u128 binom_wide(const ulonglong2* __restrict__ t, int n, int k)
{
    const ulonglong2 v = __ldg(t + n * (MAX_L + 1) + k);
    return (u128(v.y) << 64) | u128(v.x);
}
__device__ __forceinline__ uint4 wide_words(u128 k)
{
    return make_uint4(uint32_t(k), uint32_t(k >> 32), uint32_t(k >> 64), uint32_t(k >> 96));
}
__device__ __forceinline__ u128 wide_value(uint4 w)
{
    return (u128(w.w) << 96) | (u128(w.z) << 64) | (u128(w.y) << 32) | u128(w.x);
}
__device__ __forceinline__ bool wide_eq(uint4 a, uint4 b) { return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w; }

// Slot of a cone id in the open-addressing table: the 64-bit finaliser of
// SplitMix64 (Steele, Lea and Flood, 2014) over the folded words.
__device__ __forceinline__ uint32_t cone_hash(uint4 w)
{
    uint64_t h = (uint64_t(w.y) << 32 | w.x) ^ ((uint64_t(w.w) << 32 | w.z) * 0x9E3779B97F4A7C15ull);
    h ^= h >> 30;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 31;
    return uint32_t(h);
}
constexpr uint32_t HASH_EMPTY = 0xFFFFFFFFu;

// Compact cone of a 128-bit id: the table (capacity hmask + 1, a power of
// two at least twice the occupied cones, linear probing) holds the compact
// index of each occupied cone; an id that no point carries maps to
// `sentinel`, a compact cone with no rows.
__device__ __forceinline__ uint32_t cone_lookup(uint4 key, const uint4* __restrict__ ukeys,
                                                const uint32_t* __restrict__ htab, uint32_t hmask, uint32_t sentinel)
{
    uint32_t h = cone_hash(key) & hmask;
    for (uint32_t it = 0; it <= hmask; ++it) {
        const uint32_t v = __ldg(htab + h);
        if (v == HASH_EMPTY) break;
        if (wide_eq(__ldg(ukeys + v), key)) return v;
        h = (h + 1) & hmask;
    }
    return sentinel;
}

// Squared distances are >= 0, so their IEEE bit patterns order like the
// values; packing (dist bits, id) into a u64 makes u64 order the
// lexicographic (distance, id) order used for every top-k in this library.
__device__ __forceinline__ uint64_t pack_di(float d, uint32_t id)
{
    return (uint64_t(__float_as_uint(d)) << 32) | uint64_t(id);
}
constexpr uint64_t EMPTY_DI = (uint64_t(0x7F800000u) << 32) | 0xFFFFFFFFull;
__device__ __forceinline__ float di_dist(uint64_t v) { return __uint_as_float(uint32_t(v >> 32)); }
__device__ __forceinline__ uint32_t di_id(uint64_t v) { return uint32_t(v & 0xFFFFFFFFull); }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m, unsigned mask = 0xffffffffu)
{
    uint32_t lo = __shfl_xor_sync(mask, uint32_t(v), m);
    uint32_t hi = __shfl_xor_sync(mask, uint32_t(v >> 32), m);
    return (uint64_t(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        uint64_t o = shfl_xor_u64(v, m);
        v = o < v ? o : v;
    }
    return v;
}

// Register-resident top-k of packed (dist, id) keys, ascending, KMAX slots.
// For k < KMAX the first KMAX-k slots are pinned at 0 (never displaced, never
// reported), so the current k-th best is always list[KMAX-1] and no runtime
// index touches the array (it stays in registers).
template <int KMAX>
__device__ __forceinline__ void topk_init(uint64_t (&list)[KMAX], int k)
{
#pragma unroll
    for (int j = 0; j < KMAX; ++j) list[j] = j < KMAX - k ? 0ull : EMPTY_DI;
}

// Insert v; caller has checked v < list[KMAX-1].
template <int KMAX>
__device__ __forceinline__ void topk_insert(uint64_t (&list)[KMAX], uint64_t v)
{
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
        const uint64_t prev = list[j - 1];
        if (prev > v) list[j] = prev;
        else if (list[j] > v) list[j] = v;
    }
    if (list[0] > v) list[0] = v;
}

// Smallest live entry (EMPTY_DI if none).
template <int KMAX>
__device__ __forceinline__ uint64_t topk_head(const uint64_t (&list)[KMAX], int k)
{
    uint64_t m = EMPTY_DI;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j >= KMAX - k && list[j] < m) m = list[j];
    return m;
}

template <int KMAX>
__device__ __forceinline__ void topk_remove(uint64_t (&list)[KMAX], int k, uint64_t v)
{
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j >= KMAX - k && list[j] == v) list[j] = EMPTY_DI;
}

// Canonical fp32 squared distance.  The padded vector is cut into float4
// pieces j = 0 .. d_pad/4-1; piece j contributes
//     c_j = fma(t3,t3, fma(t2,t2, fma(t1,t1, t0*t0))),  t = x - y,
// and the pieces are summed as a perfect binary tree pairing adjacent
// pieces first.  Every kernel (plain scan, batched tile scan, linear search)
// evaluates exactly this expression, whatever the thread mapping, so the
// three paths return bit-identical distances for the same pair.
__device__ __forceinline__ float sq4(const float4 x, const float4 y)
{
    const float t0 = x.x - y.x, t1 = x.y - y.y, t2 = x.z - y.z, t3 = x.w - y.w;
    return fmaf(t3, t3, fmaf(t2, t2, fmaf(t1, t1, t0 * t0)));
}

// adjacent-pairwise tree over NF (power of two) pieces held by one thread
template <int NF>
__device__ __forceinline__ float pair_tree(float (&c)[NF])
{
#pragma unroll
    for (int w = 1; w < NF; w <<= 1)
#pragma unroll
        for (int j = 0; j < NF; j += 2 * w) c[j] += c[j + w];
    return c[0];
}

// continue the tree across the `lanes` (power of two) adjacent lanes that
// hold consecutive blocks of pieces
__device__ __forceinline__ float lane_tree(float v, int lanes)
{
    for (int o = 1; o < lanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ mbarrier / TMA

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking probe of the phase (mbarrier.test_wait returns at once).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// About one second at GB300 clocks: no legitimate wait here comes close.
constexpr long long WAIT_BUDGET_CYCLES = 2000000000LL;

// Wait for the phase with the given parity to complete, for at most `budget`
// SM clock cycles; false when the budget ran out.  try_wait may suspend the
// thread inside the hardware until the phase completes, so a budget shorter
// than the default (a test making the wait run out) polls with test_wait,
// which never blocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget = WAIT_BUDGET_CYCLES)
{
    if (budget < WAIT_BUDGET_CYCLES) {
        const long long t0 = clock64();
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > budget) return false;
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled on `bar` as transaction bytes.  Both addresses 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace osann
