// Tensor-core screening kernel: shared by the launchers of tc_scan.cu
// (checks off) and tc_scan_debug.cu (checks on).
//
// Batched candidate scan with 16-bit tensor-core screening and an exact fp32
// rerank.  The 16-bit operands are bf16 (unit roundoff u = 2^-8) or fp16
// (u = 2^-11, eight times tighter bound); for fp16 the data and queries are
// first multiplied by an exact power of two s, chosen from the largest row
// norm so that |s x|^2 <= 2^14, and all screening quantities are in those
// scaled units (distances scale by s^2, exactly).  Subnormal fp16 rounding
// adds an absolute error, covered by the terms Cabs(|x| + |q|).
//
// For a work item (cone c, group of up to 128 queries that probe it) the
// squared distances are first estimated on the 5th-generation tensor cores
// as  d~ = |q|^2 + |x|^2 - 2 q~.x~  (q~, x~ rounded to bf16, products exact,
// fp32 accumulation in TMEM), M = 128 queries x N = 128 cone rows per MMA
// group, the cone rows streamed by TMA (2-D tensor map over the bf16 copy of
// the permuted vectors, swizzled K-major tiles).  Each query keeps an upper
// bound U on its k-th best exact distance; a row survives the screen when
//     d~ - E(q, x) <= U,   E = 2 c |q| |x| + B (|q|^2 + |x|^2),
// where c bounds the 16-bit rounding of both operands plus the fp32
// accumulation (c = 2u + u^2 + K 2^-20) and B the fp32 error of
// the norms, of their bf16 hi/lo split and a cushion for the fp32 rounding of
// the exact distance.  The per-row terms are folded into the product by one
// extra K block of 16 columns: the query side holds (1, 1, -A', -A') with
// A' >= 2c|q| rounded up to bf16, the row side (|x|^2 hi, lo, |x| hi, lo)
// with |x|^2 scaled by (1-B), so the accumulator is directly
//     D = (1-B)|x|^2 - A'|x| - 2 q.x     and a row survives iff
//     D <= U - (1-B)|q|^2.  A
// discarded row is therefore provably farther than some candidate already
// seen, so the survivors contain the exact top-k.  Survivors are appended to
// a per-query list; the rerank computes their canonical fp32 distance (the
// same expression as every other path) and selects the top-k, so the result
// is bit-identical to the fp32 paths.  A query whose list overflows is
// rescanned in full by the rerank (counted).
#pragma once

#include <cuda.h>

#include "osann_device.cuh"
#include "osann_launch.h"
#include "osann_tc.cuh"

namespace osann {

constexpr int TC_M = 128;  // queries per item = MMA M
constexpr int TC_N = 128;  // cone rows per tile = MMA N = TMEM columns

// 16-bit conversions: PREC 0 = bf16, 1 = fp16 (round to nearest or up)
template <int PREC>
__device__ __forceinline__ uint16_t to16_rn(float f)
{
    if (PREC == 0) return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    return __half_as_ushort(__float2half_rn(f));
}
template <int PREC>
__device__ __forceinline__ uint16_t to16_ru(float f)
{
    if (PREC == 0) return __bfloat16_as_ushort(__float2bfloat16_ru(f));
    return __half_as_ushort(__float2half_ru(f));
}
template <int PREC>
__device__ __forceinline__ float from16(uint16_t h)
{
    if (PREC == 0) return __bfloat162float(__ushort_as_bfloat16(h));
    return __half2float(__ushort_as_half(h));
}
__device__ __forceinline__ uint32_t pack16(uint16_t lo, uint16_t hi) { return uint32_t(lo) | (uint32_t(hi) << 16); }

__host__ __device__ inline int tc_row_bytes(int d_pad) { return d_pad >= 64 ? 128 : d_pad * 2; }
__host__ __device__ inline int tc_kblocks(int d_pad) { return d_pad >= 64 ? d_pad / 64 : 1; }
// tile stages and query buffers per CTA: two CTAs per SM (each with its own
// MMA issuer) while the shared memory allows, else one.  Two query buffers
// suffice (a third measured no faster at d = 32); the shared memory they
// leave buys a third cone-tile stage at d = 64 (6% faster on 4096-query
// batches), the stage ring being what the producer waits on.
__host__ inline int tc_stages(int d_pad) { return d_pad <= 16 ? 6 : (d_pad == 32 ? 4 : 3); }
__host__ inline int tc_abufs(int) { return 2; }
// (both within TC_STAGES_MAX and TC_NA_MAX, the sizes of the kernel's barrier arrays)

struct TcArgs {
    const uint32_t* offsets;
    const uint32_t* perm;
    const float4* rowstat;    // per row: ((1-B)|x|^2, |x|, |x|^2, 0); N + TC_N rows
    const uint16_t* Y16;      // Q x d_pad, 16-bit -2 s y
    const float4* qstat;      // per query, scaled: (|q|^2, |q|, -A' (16-bit value, A' >= 2c|q| + Cabs), Cabs |q|)
    const float* tcs;         // (s, s^2, 1/s^2, X): X bounds every row norm (unscaled)
    const int64_t* query_src;
    const uint4* items;  // (first row, end row, first slot, slot count)
    const uint32_t* n_items_dev;
    const uint32_t* qcount;
    const uint32_t* qoff;
    const uint32_t* qlist;
    uint32_t* counter;
    uint32_t* Ubits;     // per query: upper bound on the k-th best distance (float bits)
    uint32_t* surv_cnt;  // per query
    uint32_t* surv;      // Q x cap rows
    uint32_t* status;
    unsigned long long* diag;  // [0] survivors, [1] fallbacks, [2] bound checks, [3] bound violations
    const float* xs;
    const float* Y;
    int64_t S;
    int64_t grid_w;
    int d, d_pad, k, radius, cap, stages, abufs, debug;
    float cdot2;  // 2c
    float Bn;     // B
    float cabs;   // coefficient of the subnormal rounding terms
};

// Item descriptor passed from the producer warp to the MMA and epilogue warps.
struct TcItem {
    uint32_t r0, r1;    // cone rows; r0 == 0xFFFFFFFF marks the end of the work
    uint32_t qbeg, qn;  // slot-list range of the query group
};

// Warp roles (256 threads): warp 0 lane 0 fetches items and streams the cone
// tiles with TMA; warp 1 lane 0 issues the MMAs (warp 1 owns the TMEM
// allocation); warps 2-3 ("loaders", 64 threads) gather the query tile of each
// item (asynchronous 16-byte copies of the queries' 16-bit rows straight into
// the swizzled tile) and write the per-query constants into one of the
// shared query buffers, ahead of the MMAs; warps 4-7 (128 threads, one per query row and TMEM lane)
// screen the accumulators.  Hand-offs are mbarriers: item queue (4 slots, the
// producer one item ahead of its tiles), tile stages (full/empty), query
// buffers (full/empty), accumulators (2 TMEM buffers of 128 columns,
// full/empty), so the MMA of one tile overlaps the screening of the previous
// one and the query loads overlap both.  Every wait is bounded; a timeout
// sets ST_TIMEOUT and makes all roles drop out.
//
// AT (query tiles in tensor memory; one CTA per SM, 384 threads): the query
// tile of an item is written into TMEM next to the two accumulators (lane m =
// query row m, 16-bit elements packed two per column) by warps 8-11, one
// thread per query row, and every MMA takes A from there.  The MMAs then read
// only the cone tiles from shared memory, and the shared memory of the query
// tiles holds more cone-tile stages.  Warps 2-3 idle.
constexpr int TC_ROLE_THREADS = 256;
constexpr int TC_AT_THREADS = 384;
constexpr int TC_IQ = 4;
constexpr int TC_SBUF = 8;  // survivors buffered per thread before a flush
constexpr int TC_NA_MAX = 2;
constexpr int TC_STAGES_MAX = 8;
// TMEM accumulators of TC_N columns per CTA (two CTAs share an SM's 512
// columns; a CTA alone on its SM with four was measured slower)
constexpr uint32_t TC_NACC = 2;

// per-query constants of a query tile, written by the loaders
struct TcQConst {
    float qn2;   // |q|^2 (scaled)
    float Uthr;  // s^2 U - (1-B)|q|^2 + Cq (scaled)
    float Aq1;   // A' (scaled)
    float U;     // upper bound on the k-th best exact distance (unscaled)
    float Cq;    // Cabs |q| (scaled)
    float Uoff;  // (1+B)|q|^2 + 2B s^2 X^2 + 2A' s X + Cq, X >= every row norm (scaled)
};

// DEBUG: check every screened value against an fp32 evaluation of the
// folded product (a separate instantiation, so the check costs nothing when off)
template <int KMAX, bool EXCL, int PREC, bool DEBUG, bool AT>
__global__ void __launch_bounds__(AT ? TC_AT_THREADS : TC_ROLE_THREADS, AT ? 1 : 2)
    tc_scan_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_x,
                   const TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t iq_full[TC_IQ], iq_empty[TC_IQ];
    __shared__ __align__(8) uint64_t bfull[TC_STAGES_MAX], bempty[TC_STAGES_MAX];
    __shared__ __align__(8) uint64_t afull[TC_NA_MAX], aempty[TC_NA_MAX], accfull[TC_NACC], accempty[TC_NACC];
    __shared__ TcItem iq[TC_IQ];
    __shared__ TcQConst qc[TC_NA_MAX][TC_M];
    __shared__ uint32_t qidx[TC_NA_MAX][TC_M];  // query index, 0xFFFFFFFF for an unused row
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ uint32_t sbuf_row[TC_SBUF * 128];  // survivors buffered per screening thread
    __shared__ float sbuf_val[TC_SBUF * 128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row_bytes = tc_row_bytes(a.d_pad);
    const int kblocks = tc_kblocks(a.d_pad);
    const int epb = row_bytes / 2;
    const int ksteps_pb = epb / 16;
    const int mainA = TC_M * a.d_pad * 2, mainB = TC_N * a.d_pad * 2;
    const int extA = TC_M * 32, extB = TC_N * 32;  // extra K block: 16 bf16 per row
    const int S = a.stages;
    const uint32_t NA = uint32_t(a.abufs);
    constexpr uint32_t NACC = TC_NACC;
    unsigned char* sA = base;                                       // NA x (mainA + extA); none with AT
    unsigned char* sB = AT ? base : base + NA * size_t(mainA + extA);  // S x (mainB + extB)
    // AT: TMEM columns of a query tile (d_pad / 2 packed pairs, then the 8 of the extra block)
    const uint32_t acols = uint32_t(a.d_pad / 2 + 8);
    constexpr uint32_t TMEM_COLS = AT ? 512u : NACC * TC_N;
    const uint32_t idesc = idesc_f16_f32(TC_M, TC_N, PREC == 0 ? 1u : 0u);
    const uint32_t tx_bytes = uint32_t(mainB + extB);
    const float sc = a.tcs[0], sc2 = a.tcs[1], inv_sc2 = a.tcs[2], xmax = a.tcs[3];
    // k = 1 without exclusion: the minimum of a full chunk bounds the best
    // candidate directly, and survivors need only their row
    constexpr bool FAST = KMAX == 1 && !EXCL;

    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < TC_IQ; ++i) {
            mbar_init(&iq_full[i], 1);
            // MMA issuer, 64 loader threads (4 loader warps with AT), 4 screening warps
            mbar_init(&iq_empty[i], AT ? 1 + 4 + 4 : 1 + 64 + 4);
        }
        for (int s = 0; s < S; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (uint32_t b = 0; b < NA; ++b) {
            mbar_init(&afull[b], AT ? 4 : 64);
            mbar_init(&aempty[b], 4);  // one arrival per screening warp
        }
        for (uint32_t b = 0; b < NACC; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 4);
        }
        fence_mbar_init();
        abort_sh = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_sh) return false;
        if (mbar_wait_bounded(bar, parity)) return true;
        if (!abort_sh) atomicOr(a.status, ST_TIMEOUT);
        abort_sh = 1;
        return false;
    };
    // per-query constants of a query row from its statistics and bound
    auto make_qc = [&](const float4& qsv, float Uv) -> TcQConst {
        TcQConst c;
        c.qn2 = qsv.x;
        c.U = Uv;
        c.Cq = qsv.w;
        c.Uthr = sc2 * Uv - (1.0f - a.Bn) * qsv.x + qsv.w;
        c.Aq1 = -qsv.z;
        c.Uoff = (1.0f + a.Bn) * qsv.x + 2.0f * a.Bn * sc2 * xmax * xmax + 2.0f * c.Aq1 * sc * xmax + qsv.w;
        return c;
    };

    if (warp == 0) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            const uint32_t n_items = *a.n_items_dev;
            uint32_t it = 0, tc = 0, s = 0, s_ph = 0;
            // the next item's index and descriptor are fetched one publish
            // ahead, so their latency overlaps the current item's tiles
            uint32_t pf_item = atomicAdd(a.counter, 1u);
            uint4 pf = pf_item < n_items ? a.items[pf_item] : make_uint4(0xFFFFFFFFu, 0, 0, 0);
            auto publish = [&](TcItem& out) -> bool {
                const int slot = int(it % TC_IQ);
                if (it >= TC_IQ && !wait(&iq_empty[slot], ((it / TC_IQ) - 1) & 1u)) return false;
                TcItem d;
                d.r0 = pf.x;
                d.r1 = pf.y;
                d.qbeg = pf.z;
                d.qn = pf.w;
                if (d.r0 != 0xFFFFFFFFu) {
                    pf_item = atomicAdd(a.counter, 1u);
                    pf = pf_item < n_items ? a.items[pf_item] : make_uint4(0xFFFFFFFFu, 0, 0, 0);
                }
                iq[slot] = d;
                mbar_arrive(&iq_full[slot]);
                ++it;
                out = d;
                return d.r0 != 0xFFFFFFFFu;
            };
            TcItem cur, nxt;
            bool have = publish(cur);
            while (have && !abort_sh) {
                const bool have_next = publish(nxt);  // one item ahead of its tiles
                const int ntiles = int((cur.r1 - cur.r0 + TC_N - 1) / TC_N);
                for (int t = 0; t < ntiles; ++t, ++tc) {
                    // stage s = tc mod S, s_ph = (tc / S) & 1: wait for the stage's previous use
                    if (tc >= uint32_t(S) && !wait(&bempty[s], s_ph ^ 1u)) break;
                    const int y0 = int(cur.r0) + t * TC_N;
                    unsigned char* dst = sB + size_t(s) * (mainB + extB);
                    mbar_arrive_expect_tx(&bfull[s], tx_bytes);
                    for (int kb = 0; kb < kblocks; ++kb)
                        tma_load_2d(dst + size_t(kb) * TC_N * row_bytes, &tmap, kb * epb, y0, &bfull[s]);
                    tma_load_2d(dst + mainB, &tmap_x, 0, y0, &bfull[s]);
                    if (++s == uint32_t(S)) {
                        s = 0;
                        s_ph ^= 1u;
                    }
                }
                if (abort_sh) break;
                cur = nxt;
                have = have_next;
            }
            if (abort_sh) {
                // let the last tile issued into each stage land before shared memory goes away
                for (uint32_t g = tc > uint32_t(S) ? tc - uint32_t(S) : 0u; g < tc; ++g)
                    mbar_wait_bounded(&bfull[g % uint32_t(S)], (g / uint32_t(S)) & 1u);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const int ksteps = kblocks * ksteps_pb;  // <= 8
            // descriptors of query buffer 0 and tile stage 0; a buffer, a stage
            // and a K step add their byte offset / 16 to the 14-bit start-address
            // field, which never carries (shared memory is below 2^18 bytes)
            const uint64_t da0 = smem_desc_kmajor(smem_u32(sA), row_bytes);
            const uint64_t db0 = smem_desc_kmajor(smem_u32(sB), row_bytes);
            const uint64_t dax0 = smem_desc_kmajor(smem_u32(sA + mainA), 32);
            const uint64_t dbx0 = smem_desc_kmajor(smem_u32(sB + mainB), 32);
            const uint32_t a_step = uint32_t(mainA + extA) >> 4, b_step = uint32_t(mainB + extB) >> 4;
            uint32_t koff[8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
                koff[kk] = uint32_t((kk / ksteps_pb) * TC_M * row_bytes + (kk % ksteps_pb) * 32) >> 4;
            uint32_t it = 0, tc = 0, s = 0, s_ph = 0, ab = 0, ab_ph = 0;
            for (;;) {
                const int slot = int(it % TC_IQ);
                if (!wait(&iq_full[slot], (it / TC_IQ) & 1u)) break;
                const TcItem d = iq[slot];
                if (d.r0 == 0xFFFFFFFFu) break;
                if (!wait(&afull[ab], ab_ph)) break;
                const int ntiles = int((d.r1 - d.r0 + TC_N - 1) / TC_N);
                const uint64_t da = da0 + ab * a_step, dax = dax0 + ab * a_step;
                const uint32_t ta = tmem + NACC * TC_N + ab * acols;  // AT: the query tile's columns
                bool ok = true;
                for (int t = 0; t < ntiles; ++t, ++tc) {
                    const uint32_t acc = tc % NACC;
                    if (!wait(&bfull[s], s_ph)) { ok = false; break; }
                    if (tc >= NACC && !wait(&accempty[acc], ((tc / NACC) - 1) & 1u)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t db = db0 + s * b_step, dbx = dbx0 + s * b_step;
                    const uint32_t dt = tmem + acc * TC_N;
                    if (AT) {
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            if (kk < ksteps) mma_f16_ts(dt, ta + uint32_t(kk) * 8u, db + koff[kk], idesc, kk > 0 ? 1u : 0u);
                        mma_f16_ts(dt, ta + uint32_t(a.d_pad / 2), dbx, idesc, 1u);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            if (kk < ksteps) mma_bf16_ss(dt, da + koff[kk], db + koff[kk], idesc, kk > 0 ? 1u : 0u);
                        // extra K block: |x|^2 and |x| terms folded into the product
                        mma_bf16_ss(dt, dax, dbx, idesc, 1u);
                    }
                    mma_commit(&bempty[s]);
                    mma_commit(&accfull[acc]);
                    if (++s == uint32_t(S)) {
                        s = 0;
                        s_ph ^= 1u;
                    }
                }
                if (!ok) break;
                mbar_arrive(&iq_empty[slot]);
                ++it;
                if (++ab == NA) {
                    ab = 0;
                    ab_ph ^= 1u;
                }
            }
            if (abort_sh && tc > 0) mbar_wait_bounded(&accfull[(tc - 1) % NACC], ((tc - 1) / NACC) & 1u);
        }
    } else if (!AT && warp < 4) {
        // ------------------------------------------------ query tile loaders
        // warp 2 gathers query rows 0..63 of the tile, warp 3 rows 64..127;
        // lane l holds the indices and constants of rows rb + l and rb + 32 + l
        const int rb = 64 * (warp - 2);
        const int cpr = a.d_pad / 8;  // 16-byte chunks per 16-bit query row (2, 4, 8 or 16)
        const int cpr_sh = __ffs(cpr) - 1;
        const int chunks_sh = __ffs(row_bytes / 16) - 1;  // chunks per row of one K block of the tile
        for (uint32_t it = 0;; ++it) {
            const int slot = int(it % TC_IQ);
            if (!wait(&iq_full[slot], (it / TC_IQ) & 1u)) break;
            const TcItem d = iq[slot];
            if (d.r0 == 0xFFFFFFFFu) break;
            const uint32_t ab = it % NA;
            if (it >= NA && !wait(&aempty[ab], ((it / NA) - 1) & 1u)) break;
            unsigned char* dstA = sA + size_t(ab) * (mainA + extA);
            // both rows' query indices; then the warp's 64 16-bit rows as
            // asynchronous 16-byte copies straight into the swizzled tile, every
            // chunk in flight at once, consecutive lanes on consecutive chunks of
            // one row (each instruction reads whole 32-byte sectors); while those
            // land, both rows' constants
            uint32_t qr[2];
            float4 qs[2];
            float Ur[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = rb + lane + 32 * h;
                qr[h] = uint32_t(r) < d.qn ? a.qlist[d.qbeg + r] / uint32_t(a.S) : 0xFFFFFFFFu;
            }
            for (int j = 0; j < 2 * cpr; ++j) {
                const int i = lane + 32 * j;  // chunk of the warp's rows
                const int rl = i >> cpr_sh, ch = i & (cpr - 1);
                // rl < 32 for all lanes or for none: the source register is uniform
                const uint32_t qs_src = __shfl_sync(0xffffffffu, j < cpr ? qr[0] : qr[1], rl & 31);
                unsigned char* dst = dstA + size_t(ch >> chunks_sh) * TC_M * row_bytes +
                                     swz_offset(rb + rl, ch & ((1 << chunks_sh) - 1), row_bytes);
                if (qs_src != 0xFFFFFFFFu)
                    cp_async16(dst, reinterpret_cast<const uint4*>(a.Y16 + int64_t(qs_src) * a.d_pad) + ch);
                else
                    *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                qs[h] = make_float4(0.f, 0.f, 0.f, 0.f);
                Ur[h] = INFINITY;
                if (qr[h] != 0xFFFFFFFFu) {
                    qs[h] = a.qstat[qr[h]];
                    Ur[h] = __uint_as_float(a.Ubits[qr[h]]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = rb + lane + 32 * h;
                const bool active = qr[h] != 0xFFFFFFFFu;
                // extra block: (1, 1, -A', -A', 0, ...) against (|x|^2 hi, lo, |x| hi, lo, 0, ...)
                uint4 e0 = make_uint4(0, 0, 0, 0);
                if (active) {
                    const uint16_t one = to16_rn<PREC>(1.0f), na = to16_rn<PREC>(qs[h].z);  // exact
                    e0.x = pack16(one, one);
                    e0.y = pack16(na, na);
                }
                *reinterpret_cast<uint4*>(dstA + mainA + swz_offset(r, 0, 32)) = e0;
                *reinterpret_cast<uint4*>(dstA + mainA + swz_offset(r, 1, 32)) = make_uint4(0, 0, 0, 0);
                qc[ab][r] = make_qc(qs[h], Ur[h]);
                qidx[ab][r] = qr[h];
            }
            // this thread's copies have landed; make them and the stores above
            // visible to the tensor core (async proxy)
            cp_async_wait_all();
            fence_proxy_async_smem();
            mbar_arrive(&afull[ab]);
            mbar_arrive(&iq_empty[slot]);
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ screening
        const int er = 32 * (warp & 3) + lane;  // query row of the group = TMEM lane
        const uint32_t tl = tmem + (uint32_t(32 * (warp & 3)) << 16);
        for (uint32_t it = 0, tc = 0;; ++it) {
            const int slot = int(it % TC_IQ);
            if (!wait(&iq_full[slot], (it / TC_IQ) & 1u)) break;
            const TcItem dc = iq[slot];
            if (dc.r0 == 0xFFFFFFFFu) break;
            const uint32_t ab = it % NA;
            if (!wait(&afull[ab], (it / NA) & 1u)) break;
            TcQConst cur = qc[ab][er];
            const float U0 = cur.U;
            const uint32_t qi = qidx[ab][er];
            const bool active = qi != 0xFFFFFFFFu;
            const int64_t q = active ? int64_t(qi) : 0;
            const int64_t src = EXCL && active ? a.query_src[q] : -1;
            const int ntiles = int((dc.r1 - dc.r0 + TC_N - 1) / TC_N);
            float ubl[KMAX];  // k smallest upper bounds seen for this query in this item
#pragma unroll
            for (int u = 0; u < KMAX; ++u) ubl[u] = INFINITY;
            int nb = 0;  // survivors buffered in shared memory by this thread
            // append the buffered survivors (minus excluded rows) to the query's
            // list, then tighten U with their upper bounds (deferred: a stale U
            // only admits more rows)
            auto flush = [&]() {
                if (FAST) {
                    if (nb > 0) {
                        const uint32_t pos = atomicAdd(a.surv_cnt + q, uint32_t(nb));
                        for (int i = 0; i < nb; ++i)
                            if (pos + uint32_t(i) < uint32_t(a.cap)) a.surv[q * a.cap + pos + i] = sbuf_row[i * 128 + er];
                    }
                    nb = 0;
                    return;
                }
                int keep = 0;
                for (int i = 0; i < nb; ++i) {
                    const uint32_t row = sbuf_row[i * 128 + er];
                    if (EXCL && src >= 0) {
                        const int64_t id = int64_t(__ldg(a.perm + row));
                        int64_t dr = id / a.grid_w - src / a.grid_w, dcc = id % a.grid_w - src % a.grid_w;
                        dr = dr < 0 ? -dr : dr;
                        dcc = dcc < 0 ? -dcc : dcc;
                        if ((dr > dcc ? dr : dcc) <= a.radius) continue;
                    }
                    sbuf_row[keep * 128 + er] = row;
                    sbuf_val[keep * 128 + er] = sbuf_val[i * 128 + er];
                    ++keep;
                }
                if (keep > 0) {
                    const uint32_t pos = atomicAdd(a.surv_cnt + q, uint32_t(keep));
                    for (int i = 0; i < keep; ++i) {
                        const uint32_t row = sbuf_row[i * 128 + er];
                        const float D = sbuf_val[i * 128 + er];
                        if (pos + uint32_t(i) < uint32_t(a.cap)) a.surv[q * a.cap + pos + i] = row;
                        // d~ + E <= D + (1+B)|q|^2 + 2B|x|^2 + 2A'|x| + Cq (scaled units)
                        const float4 rs = __ldg(a.rowstat + row);
                        const float ubs = (D + (1.0f + a.Bn) * cur.qn2 + 2.0f * a.Bn * sc2 * rs.z +
                                           2.0f * cur.Aq1 * sc * rs.y + cur.Cq) * (1.0f + 1e-6f);
                        const float ub = fmaxf(ubs * inv_sc2, 0.0f);
                        if (ub < ubl[KMAX - 1]) {
#pragma unroll
                            for (int u = KMAX - 1; u > 0; --u) {
                                const float pu = ubl[u - 1];
                                if (pu > ub) ubl[u] = pu;
                                else if (ubl[u] > ub) ubl[u] = ub;
                            }
                            if (ubl[0] > ub) ubl[0] = ub;
                        }
                    }
                    // the k-th smallest bound of k distinct candidates bounds the k-th best
                    float kth = INFINITY;
#pragma unroll
                    for (int u = 0; u < KMAX; ++u)
                        if (u == a.k - 1) kth = ubl[u];
                    if (kth < cur.U) {
                        cur.U = kth;
                        cur.Uthr = sc2 * cur.U - (1.0f - a.Bn) * cur.qn2 + cur.Cq;
                    }
                }
                nb = 0;
            };
            bool ok = true;
            for (int t = 0; t < ntiles; ++t, ++tc) {
                const int acc = int(tc % NACC);
                if (!wait(&accfull[acc], (tc / NACC) & 1u)) { ok = false; break; }
                tc_fence_after();
                const int y0 = int(dc.r0) + t * TC_N;
                const int nvalid = min(TC_N, int(dc.r1) - y0);
                for (int c0 = 0; c0 < nvalid; c0 += 64) {
                    float v[64], m[2];
                    tmem_ld32x2_min(tl + uint32_t(acc * TC_N + c0), v, m[0], m[1]);
                    const float vmin = fminf(m[0], m[1]);
                    const int lim = nvalid - c0;
                    // columns past the item's rows (the next cone's, in the last
                    // tile) can only lower the minimum: the exact mask below drops them
                    if (active && vmin <= cur.Uthr) {
                        if (FAST && lim >= 64) {
                            // every column is a row of the item's cone, so the row at
                            // the minimum is a candidate within this bound
                            const float ub = fmaxf((vmin + cur.Uoff) * (1.0f + 1e-6f) * inv_sc2, 0.0f);
                            if (ub < cur.U) {
                                cur.U = ub;
                                cur.Uthr = sc2 * cur.U - (1.0f - a.Bn) * cur.qn2 + cur.Cq;
                            }
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            uint32_t mask = 0;
#pragma unroll
                            for (int j = 0; j < 32; ++j) mask |= (v[32 * h + j] <= cur.Uthr ? 1u : 0u) << j;
                            // a masked column is +inf, which an unbounded U would admit
                            const int limh = lim - 32 * h;
                            if (limh < 32) mask &= limh <= 0 ? 0u : (1u << limh) - 1u;
                            while (mask) {
                                const int j = __ffs(int(mask)) - 1;
                                mask &= mask - 1u;
                                if (nb == TC_SBUF) flush();
                                sbuf_row[nb * 128 + er] = uint32_t(y0 + c0 + 32 * h + j);
                                if (!FAST) {
                                    float val = v[32 * h];
#pragma unroll
                                    for (int u = 1; u < 32; ++u) val = u == j ? v[32 * h + u] : val;
                                    sbuf_val[nb * 128 + er] = val;
                                }
                                ++nb;
                            }
                        }
                    }
                    if (DEBUG && active) {
                        // folded product against an fp32 evaluation, one column per thread
                        const int col = lane + 32 * (c0 / 64 % 2);
                        if (col < lim) {
                            const int row = y0 + c0 + col;
                            const float* xr = a.xs + size_t(row) * a.d_pad;
                            const float* yr = a.Y + q * int64_t(a.d);
                            float dot = 0.f;
                            for (int i = 0; i < a.d; ++i) dot = fmaf(xr[i], yr[i], dot);
                            const float4 rs = __ldg(a.rowstat + row);
                            float mine = v[0];
#pragma unroll
                            for (int u = 1; u < 64; ++u) mine = u == col ? v[u] : mine;
                            const float ref = -2.0f * sc2 * dot + sc2 * rs.x - cur.Aq1 * sc * rs.y;
                            const float qnorm = sqrtf(cur.qn2);
                            const float lim2 = a.cdot2 * qnorm * sc * rs.y * 1.001f +
                                               4.0f * a.Bn * (cur.qn2 + sc2 * rs.z) +
                                               2.0f * a.cabs * (sc * rs.y + qnorm) + 1e-30f;
                            atomicAdd(a.diag + 2, 1ull);
                            if (fabsf(mine - ref) > lim2) {
                                atomicAdd(a.diag + 3, 1ull);
                                atomicOr(a.status, ST_BOUND);
                            }
                        }
                    }
                }
                // every lane's loads of this accumulator are complete: one arrival per warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&accempty[acc]);
            }
            if (!ok) break;
            if (active) {
                flush();
                if (cur.U < U0) atomicMin(a.Ubits + q, __float_as_uint(fmaxf(cur.U, 0.0f)));
            }
            // the warp has read its query constants and the item descriptor
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&aempty[ab]);
                mbar_arrive(&iq_empty[slot]);
            }
        }
    } else if (AT && warp >= 8) {
        // ------------------------------------------------ query tiles into TMEM (AT, d_pad = 128)
        const int r = 32 * (warp & 3) + lane;  // query row of the tile = TMEM lane
        const uint32_t tl = tmem + (uint32_t(32 * (warp & 3)) << 16);
        const int cpr = a.d_pad / 8;  // 16-byte chunks of a 16-bit query row (16)
        for (uint32_t it = 0;; ++it) {
            const int slot = int(it % TC_IQ);
            if (!wait(&iq_full[slot], (it / TC_IQ) & 1u)) break;
            const TcItem d = iq[slot];
            if (d.r0 == 0xFFFFFFFFu) break;
            const uint32_t ab = it % NA;
            if (it >= NA && !wait(&aempty[ab], ((it / NA) - 1) & 1u)) break;
            // the MMAs that read this buffer's columns have completed
            tc_fence_after();
            const uint32_t qr = uint32_t(r) < d.qn ? a.qlist[d.qbeg + r] / uint32_t(a.S) : 0xFFFFFFFFu;
            const bool active = qr != 0xFFFFFFFFu;
            const uint4* src = reinterpret_cast<const uint4*>(a.Y16 + int64_t(active ? qr : 0u) * a.d_pad);
            uint4 row[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) row[c] = active && c < cpr ? __ldg(src + c) : make_uint4(0, 0, 0, 0);
            float4 qs = make_float4(0.f, 0.f, 0.f, 0.f);
            float Ur = INFINITY;
            uint4 e0 = make_uint4(0, 0, 0, 0);
            if (active) {
                qs = a.qstat[qr];
                Ur = __uint_as_float(a.Ubits[qr]);
                // extra block: (1, 1, -A', -A', 0, ...) against (|x|^2 hi, lo, |x| hi, lo, 0, ...)
                const uint16_t one = to16_rn<PREC>(1.0f), na = to16_rn<PREC>(qs.z);  // exact
                e0.x = pack16(one, one);
                e0.y = pack16(na, na);
            }
            qc[ab][r] = make_qc(qs, Ur);
            qidx[ab][r] = qr;
            const uint32_t tcol = tl + NACC * TC_N + ab * acols;
            tmem_st64(tcol, row);
            tmem_st8(tcol + uint32_t(a.d_pad / 2), e0, make_uint4(0, 0, 0, 0));
            // the tile's columns are written; order them before the MMAs
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&afull[ab]);
                mbar_arrive(&iq_empty[slot]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// AT: cone-tile stages in the shared memory the query tiles leave (d_pad = 128:
// five of 36 KB)
__host__ inline int tc_stages_at(int d_pad) { return d_pad == 128 ? 5 : tc_stages(d_pad); }

inline size_t tc_smem_bytes(int d_pad, bool at)
{
    const size_t tileA = size_t(TC_M) * d_pad * 2 + TC_M * 32, tileB = size_t(TC_N) * d_pad * 2 + TC_N * 32;
    if (at) return 1024 + size_t(tc_stages_at(d_pad)) * tileB;
    const size_t need = 1024 + size_t(tc_abufs(d_pad)) * tileA + size_t(tc_stages(d_pad)) * tileB;
    // at least 80 KB so that at most two CTAs (2 x 256 TMEM columns) share an SM
    return need < 80u * 1024u ? 80u * 1024u : need;
}

template <int KMAX, bool EXCL, int PREC, bool DEBUG, bool AT = false>
static int launch_tc_t(const void* maps, const TcArgs& a, cudaStream_t st, int num_sms)
{
    const size_t smem = tc_smem_bytes(a.d_pad, AT);
    auto kern = tc_scan_kernel<KMAX, EXCL, PREC, DEBUG, AT>;
    constexpr int threads = AT ? TC_AT_THREADS : TC_ROLE_THREADS;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    // resident CTAs per SM: registers, shared memory (228 KB per SM, 1 KB
    // reserved per CTA) and TMEM (512 columns: 256 per CTA, all of them with AT)
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kern);
    const int regs = fa.numRegs > 0 ? fa.numRegs : 255;
    const int by_regs = 65536 / (regs * threads);
    const int by_smem = int((228u * 1024u) / (smem + 1024u + size_t(fa.sharedSizeBytes)));
    int occ = by_regs < by_smem ? by_regs : by_smem;
    if (occ > (AT ? 1 : 2)) occ = AT ? 1 : 2;
    if (occ < 1) occ = 1;
    cudaGetLastError();
    const CUtensorMap* m = static_cast<const CUtensorMap*>(maps);
    kern<<<unsigned(num_sms * occ), threads, smem, st>>>(m[0], m[1], a);
    return count_launch();
}

// tc_scan_tmem.cu: the launches with the query tiles in TMEM (d_pad = 128,
// no exclusion), bound check on or off
int launch_tc_scan_tmem(const void* maps, const TcArgs& a, int k, int prec, bool debug, cudaStream_t st, int num_sms);

// tc_scan_debug.cu: the same launch with the bound check compiled in
int launch_tc_scan_debug(const void* maps, const TcArgs& a, int k, int prec, bool excl, cudaStream_t st, int num_sms);

}  // namespace osann
