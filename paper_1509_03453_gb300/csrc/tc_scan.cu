// Tensor-core screening path: query preparation (seed bounds, 16-bit query
// operands), the fp16 scale and row operands, tensor maps, the screening
// launch (kernel in tc_scan_kernel.cuh) and the exact fp32 rerank.
#include "osann.h"
#include "tc_scan_kernel.cuh"

namespace osann {

// ---------------------------------------------------------------- query prep

// One warp per query: 16-bit copy of -2 s y, scaled norms and A', survivor
// counter reset, and the initial upper bound U: the k-th smallest canonical
// fp32 distance over the rows of the first probed cones (in probe order,
// excluded rows skipped, at least `seed_rows` rows when the cones hold them),
// inflated by the fp32 error bound; +inf if fewer than k rows.  A query too large for the 16-bit range is left to the
// rerank's full scan (its survivor count is set above the capacity).
constexpr int TC_SEED_ILP = 8;  // row groups loaded per iteration

// Rows scanned exactly for a query's initial bound.  A large batch keeps
// tightening its bounds as items finish, so a short seed suffices (64 rows
// from 4096 queries up; measured on 4096-query batches of d = 64 and 128,
// 64 rows halve this kernel's time and cost the screen and rerank less than
// that); in a small batch every item runs at once on the first bound, which
// must then be tighter (up to 1024 rows, a few cones): about 2^18 / Q rows,
// clamped.  For k > 4 the bound is the k-th best of the seed, which a short
// seed leaves loose: 1024 rows (on the thin-cone descriptor search, k = 10,
// Q = 10^4, this cut the survivors from 9.7 to 2.0 million and removed the
// overflow rescans: 26.2 -> 21.5 ms).
static int tc_seed_rows(int64_t Q, int k)
{
    if (k > 4) return 1024;
    const int64_t r = Q > 0 ? (int64_t(262144) + Q - 1) / Q : 1024;
    return int(r < 64 ? 64 : (r > 1024 ? 1024 : r));
}

template <int F, int PREC, int KMAX>
__global__ void __launch_bounds__(128) tc_query_prep_kernel(const float* __restrict__ Y, int64_t Q, int d, int d_pad,
                                                            const uint32_t* __restrict__ probes, int64_t P_eff,
                                                            const uint32_t* __restrict__ offsets, uint32_t NC,
                                                            const float* __restrict__ xs, int k, float cdot2,
                                                            float cabs, const float* __restrict__ tcs,
                                                            const uint32_t* __restrict__ perm,
                                                            const int64_t* __restrict__ query_src, int64_t grid_w,
                                                            int radius, int cap, uint16_t* __restrict__ Y16,
                                                            float4* __restrict__ qstat, uint32_t* __restrict__ Ubits,
                                                            uint32_t* __restrict__ surv_cnt, int seed_rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;  // whole warp
    const float* y = Y + q * int64_t(d);
    const float sc = tcs[0];
    float s = 0.f, amax = 0.f;
    for (int c = lane * 4; c < d_pad; c += 128) {
        float4 v;
        v.x = c + 0 < d ? y[c + 0] : 0.f;
        v.y = c + 1 < d ? y[c + 1] : 0.f;
        v.z = c + 2 < d ? y[c + 2] : 0.f;
        v.w = c + 3 < d ? y[c + 3] : 0.f;
        // -2 s y: the factor is a power of two, so the 16-bit value is exact
        // up to the 16-bit rounding of s y itself
        uint2 pk;
        pk.x = pack16(to16_rn<PREC>(-2.f * sc * v.x), to16_rn<PREC>(-2.f * sc * v.y));
        pk.y = pack16(to16_rn<PREC>(-2.f * sc * v.z), to16_rn<PREC>(-2.f * sc * v.w));
        *reinterpret_cast<uint2*>(Y16 + q * int64_t(d_pad) + c) = pk;
        s = fmaf(v.x, v.x, s);
        s = fmaf(v.y, v.y, s);
        s = fmaf(v.z, v.z, s);
        s = fmaf(v.w, v.w, s);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    // fp16 holds |v| < 65504; keep 2 |s y| and the norm terms well inside
    const bool unscreenable = PREC == 1 && (2.f * sc * amax > 16384.f || sc * sc * s > 32768.f);

    // seed rows: TPR lanes per row (canonical distance, as in the rerank)
    const int n4 = d_pad >> 2;
    const int TPR = n4 / F, CPP = 32 / TPR;
    const int g = lane / TPR, sub = lane % TPR;
    float4 qv[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const int c = 4 * (sub * F + f);
        qv[f].x = c + 0 < d ? y[c + 0] : 0.f;
        qv[f].y = c + 1 < d ? y[c + 1] : 0.f;
        qv[f].z = c + 2 < d ? y[c + 2] : 0.f;
        qv[f].w = c + 3 < d ? y[c + 3] : 0.f;
    }
    const int64_t src = query_src ? query_src[q] : -1;
    uint64_t list[KMAX];
    topk_init<KMAX>(list, k);
    int scanned = 0;
    for (int64_t p = 0; p < P_eff && scanned < seed_rows; ++p) {
        const uint32_t b = probes[q * P_eff + p];
        if (b >= NC) continue;
        const uint32_t o0 = offsets[b], o1 = offsets[b + 1];
        for (uint32_t r0 = o0; r0 < o1 && scanned < seed_rows; r0 += TC_SEED_ILP * CPP) {
            // TC_SEED_ILP row groups per iteration: all loads in flight before the arithmetic
            float4 xv[TC_SEED_ILP][F];
            uint32_t rr[TC_SEED_ILP];
#pragma unroll
            for (int u = 0; u < TC_SEED_ILP; ++u) {
                rr[u] = r0 + uint32_t(u * CPP + g);
                const float4* xr =
                    reinterpret_cast<const float4*>(xs + size_t(rr[u] < o1 ? rr[u] : o0) * d_pad) + sub * F;
#pragma unroll
                for (int f = 0; f < F; ++f) xv[u][f] = xr[f];
            }
#pragma unroll
            for (int u = 0; u < TC_SEED_ILP; ++u) {
                float cpart[F];
#pragma unroll
                for (int f = 0; f < F; ++f) cpart[f] = sq4(xv[u][f], qv[f]);
                const float dist = lane_tree(pair_tree<F>(cpart), TPR);
                bool usable = rr[u] < o1;
                if (usable && src >= 0) {
                    // an excluded row is not a candidate and cannot seed the bound
                    const int64_t id = int64_t(perm[rr[u]]);
                    int64_t dr = id / grid_w - src / grid_w, dc = id % grid_w - src % grid_w;
                    dr = dr < 0 ? -dr : dr;
                    dc = dc < 0 ? -dc : dc;
                    usable = (dr > dc ? dr : dc) > radius;
                }
                if (sub == 0 && usable) {
                    const uint64_t v = pack_di(dist, rr[u]);
                    if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                }
            }
            scanned += TC_SEED_ILP * CPP;
        }
    }
    // k-th smallest over the warp: k rounds of warp minimum over the lists
    float U = INFINITY;
    {
        float kth = INFINITY;
        int found = 0;
        for (int j = 0; j < k; ++j) {
            const uint64_t head = topk_head<KMAX>(list, k);
            const uint64_t best = warp_min_u64(head);
            if (best == EMPTY_DI) break;
            if (head == best) topk_remove<KMAX>(list, k, best);
            kth = di_dist(best);
            ++found;
        }
        // the canonical fp32 distance is within 6.6e-7 relative of the exact one
        if (found == k) U = kth * (1.0f + 2e-6f) + 1e-30f;
    }
    if (lane == 0) {
        // scaled units: |q'| = s |q|; A' = 2c|q'| + Cabs, inflated by 2^-14
        // (16-bit hi/lo split of |x|) and rounded up to the 16-bit format
        const float qn = sc * sc * s, qnorm = sc * sqrtf(s);
        const float A = (cdot2 * qnorm + cabs) * (1.0f + 6.1035156e-5f);
        const float Ap = from16<PREC>(to16_ru<PREC>(A));
        qstat[q] = make_float4(qn, qnorm, -Ap, cabs * qnorm);
        Ubits[q] = __float_as_uint(U);
        surv_cnt[q] = unscreenable ? uint32_t(cap) + 1u : 0u;
    }
}

// ---------------------------------------------------------------- rows

// The data scale of the screen: s = 1 for bf16; for fp16 the power of two
// with s^2 max|x|^2 <= 2^14 (all-zero data: 1).  tcs = (s, s^2, 1/s^2, X), X >= every row norm.
template <int PREC>
__global__ void tc_scale_kernel(const uint32_t* __restrict__ maxn2_bits, float* __restrict__ tcs)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int e = 0;
    const float m = __uint_as_float(*maxn2_bits);
    if (PREC == 1 && m > 0.0f) {
        int x;
        frexpf(m, &x);  // m < 2^x
        const int t = 14 - x;
        e = t >= 0 ? t / 2 : -((1 - t) / 2);
        e = e > 40 ? 40 : (e < -40 ? -40 : e);
    }
    const float sc = ldexpf(1.0f, e);
    tcs[0] = sc;
    tcs[1] = sc * sc;
    tcs[2] = 1.0f / (sc * sc);
    // a bound on every row norm, with room for the differently ordered fp32
    // sums of the per-row norms
    tcs[3] = sqrtf(m * (1.0f + 1e-4f)) * (1.0f + 1e-6f);
}

// 16-bit copy of s x (row-major, d_pad per row) and the extra K block of each
// row: 16-bit hi/lo splits of (1-B) s^2 |x|^2 and s |x|, then zeros.
template <int PREC>
__global__ void __launch_bounds__(256) tc_rows_kernel(const float* __restrict__ xs, const float4* __restrict__ rowstat,
                                                      int64_t N, int d_pad, const float* __restrict__ tcs,
                                                      uint16_t* __restrict__ x16, uint16_t* __restrict__ xe16)
{
    const float sc = tcs[0], sc2 = tcs[1];
    const int64_t n4 = N * (d_pad / 4);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
        const float4 v = reinterpret_cast<const float4*>(xs)[i];
        uint2 pk;
        pk.x = pack16(to16_rn<PREC>(sc * v.x), to16_rn<PREC>(sc * v.y));
        pk.y = pack16(to16_rn<PREC>(sc * v.z), to16_rn<PREC>(sc * v.w));
        reinterpret_cast<uint2*>(x16)[i] = pk;
    }
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += int64_t(gridDim.x) * blockDim.x) {
        const float4 rs = rowstat[r];
        const float a = sc2 * rs.x, b = sc * rs.y;
        const uint16_t ah = to16_rn<PREC>(a), bh = to16_rn<PREC>(b);
        const uint16_t al = to16_rn<PREC>(a - from16<PREC>(ah)), bl = to16_rn<PREC>(b - from16<PREC>(bh));
        uint4* dst = reinterpret_cast<uint4*>(xe16 + r * 16);
        dst[0] = make_uint4(pack16(ah, al), pack16(bh, bl), 0u, 0u);
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

int launch_tc_scale(int prec, const uint32_t* maxn2_bits, float* tcs, cudaStream_t st)
{
    if (prec == 0) tc_scale_kernel<0><<<1, 32, 0, st>>>(maxn2_bits, tcs);
    else tc_scale_kernel<1><<<1, 32, 0, st>>>(maxn2_bits, tcs);
    return count_launch();
}

int launch_tc_rows(int prec, const float* xs, const float4* rowstat, int64_t N, int d_pad, const uint32_t* maxn2_bits,
                   float* tcs, void* x16, void* xe16, cudaStream_t st, int num_sms)
{
    if (prec == 0) tc_scale_kernel<0><<<1, 32, 0, st>>>(maxn2_bits, tcs);
    else tc_scale_kernel<1><<<1, 32, 0, st>>>(maxn2_bits, tcs);
    int rc = count_launch();
    if (rc || N == 0) return rc;
    int64_t blocks = (N * (d_pad / 4) + 255) / 256;
    if (blocks > int64_t(num_sms) * 16) blocks = int64_t(num_sms) * 16;
    if (prec == 0)
        tc_rows_kernel<0><<<unsigned(blocks), 256, 0, st>>>(xs, rowstat, N, d_pad, tcs, static_cast<uint16_t*>(x16),
                                                             static_cast<uint16_t*>(xe16));
    else
        tc_rows_kernel<1><<<unsigned(blocks), 256, 0, st>>>(xs, rowstat, N, d_pad, tcs, static_cast<uint16_t*>(x16),
                                                             static_cast<uint16_t*>(xe16));
    return count_launch();
}

// ---------------------------------------------------------------- rerank

constexpr int RR_U = 4;  // candidate passes with their loads in flight together

// One warp per query: canonical fp32 distance of every survivor (or, after
// an overflow, of every row of every probed cone), top-k by (distance, id).
template <int F, int KMAX, bool EXCL>
__global__ void __launch_bounds__(128) tc_rerank_kernel(const float* __restrict__ xs, int d_pad,
                                                        const uint32_t* __restrict__ perm,
                                                        const uint32_t* __restrict__ offsets, uint32_t NC,
                                                        const float* __restrict__ Y, int d, int64_t Q,
                                                        const uint32_t* __restrict__ probes, int64_t P_eff,
                                                        const uint32_t* __restrict__ surv_cnt,
                                                        const uint32_t* __restrict__ surv, int cap, int k,
                                                        const int64_t* __restrict__ query_src, int64_t grid_w,
                                                        int radius, unsigned long long* __restrict__ diag,
                                                        uint32_t* __restrict__ ovf, int64_t* __restrict__ out_ids,
                                                        float* __restrict__ out_d)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const int n4 = d_pad >> 2;
    const int TPR = n4 / F;         // lanes per candidate (<= 32)
    const int CPP = 32 / TPR;       // candidates per pass
    const int g = lane / TPR, sub = lane % TPR;
    float4 qv[F];
    {
        const float* y = Y + q * int64_t(d);
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int c = 4 * (sub * F + f);
            qv[f].x = c + 0 < d ? y[c + 0] : 0.f;
            qv[f].y = c + 1 < d ? y[c + 1] : 0.f;
            qv[f].z = c + 2 < d ? y[c + 2] : 0.f;
            qv[f].w = c + 3 < d ? y[c + 3] : 0.f;
        }
    }
    const int64_t src = EXCL ? query_src[q] : -1;
    uint64_t list[KMAX];
    topk_init<KMAX>(list, k);
    // the candidate's canonical distance from its row chunk xv (this lane's F
    // float4 of the row), then the top-k update
    auto consider = [&](uint32_t row, bool valid, const float4 (&xv)[F]) {
        float cpart[F];
#pragma unroll
        for (int f = 0; f < F; ++f) cpart[f] = sq4(xv[f], qv[f]);
        const float dist = lane_tree(pair_tree<F>(cpart), TPR);
        if (valid && sub == 0) {
            const uint32_t id = __ldg(perm + row);
            if (EXCL && src >= 0) {
                const int64_t dr = int64_t(id) / grid_w - src / grid_w;
                const int64_t dc = int64_t(id) % grid_w - src % grid_w;
                const int64_t adr = dr < 0 ? -dr : dr, adc = dc < 0 ? -dc : dc;
                if ((adr > adc ? adr : adc) <= radius) return;
            }
            const uint64_t v = pack_di(dist, id);
            if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
        }
    };
    const uint32_t n = surv_cnt[q];
    if (n <= uint32_t(cap)) {
        // RR_U passes at a time: their survivor ids, then their rows, are all
        // in flight before the first distance
        for (uint32_t b0 = 0; b0 < n; b0 += RR_U * uint32_t(CPP)) {
            uint32_t rows[RR_U];
            bool valid[RR_U];
#pragma unroll
            for (int u = 0; u < RR_U; ++u) {
                const uint32_t i = b0 + uint32_t(u * CPP + g);
                valid[u] = i < n;
                rows[u] = valid[u] ? surv[q * cap + i] : 0u;
            }
            float4 xv[RR_U][F];
#pragma unroll
            for (int u = 0; u < RR_U; ++u) {
                const float4* xr = reinterpret_cast<const float4*>(xs + size_t(rows[u]) * d_pad) + sub * F;
#pragma unroll
                for (int f = 0; f < F; ++f) xv[u][f] = xr[f];
            }
#pragma unroll
            for (int u = 0; u < RR_U; ++u) consider(rows[u], valid[u], xv[u]);
        }
        if (lane == 0) atomicAdd(diag, (unsigned long long)n);
    } else {
        // survivor list overflowed: the query is rescanned by the plain scan
        if (lane == 0) {
            atomicAdd(diag + 1, 1ull);
            ovf[1 + atomicAdd(ovf, 1u)] = uint32_t(q);
        }
        return;
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

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int tc_encode_rows_map(void* map_out, const void* x16, int64_t N, int d_pad, int prec)
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult qr;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            set_error("cuTensorMapEncodeTiled is not available");
            return -2;
        }
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    // d_pad == 0 encodes the 16-column extra block array instead
    const int width = d_pad > 0 ? d_pad : 16;
    const int row_bytes = d_pad > 0 ? tc_row_bytes(d_pad) : 32;
    const cuuint64_t dims[2] = {cuuint64_t(width), cuuint64_t(N)};
    const cuuint64_t strides[1] = {cuuint64_t(width) * 2};
    const cuuint32_t box[2] = {cuuint32_t(row_bytes / 2), cuuint32_t(TC_N)};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                   : (row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                      : CU_TENSOR_MAP_SWIZZLE_32B);
    CUresult r = fn(static_cast<CUtensorMap*>(map_out),
                    prec == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    const_cast<void*>(x16), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", int(r));
        return -5;
    }
    return 0;
}

size_t tc_map_bytes() { return 2 * sizeof(CUtensorMap); }

int launch_tc_query_prep(int prec, const float* Y, int64_t Q, int d, int d_pad, const uint32_t* probes,
                         int64_t P_eff, const uint32_t* offsets, uint32_t NC, const float* xs, int k, float cdot2,
                         float cabs, const float* tcs, const uint32_t* perm, const int64_t* query_src, int64_t grid_w,
                         int radius, int cap, void* Y16, float4* qstat, uint32_t* Ubits, uint32_t* surv_cnt,
                         cudaStream_t st)
{
    if (Q == 0) return 0;
    const unsigned blocks = unsigned((Q * 32 + 127) / 128);
    uint16_t* y16 = static_cast<uint16_t*>(Y16);
    const int seed_rows = tc_seed_rows(Q, k);
#define OSANN_PREP(F, PR, KM)                                                                                       \
    tc_query_prep_kernel<F, PR, KM><<<blocks, 128, 0, st>>>(Y, Q, d, d_pad, probes, P_eff, offsets, NC, xs, k, cdot2, \
                                                            cabs, tcs, perm, query_src, grid_w, radius, cap, y16,    \
                                                            qstat, Ubits, surv_cnt, seed_rows)
#define OSANN_PREP_K(F, PR)             \
    if (k <= 1) OSANN_PREP(F, PR, 1);      \
    else if (k <= 4) OSANN_PREP(F, PR, 4); \
    else if (k <= 16) OSANN_PREP(F, PR, 16); \
    else OSANN_PREP(F, PR, 32);
    if (d_pad <= 128) {
        if (prec == 0) { OSANN_PREP_K(1, 0) }
        else { OSANN_PREP_K(1, 1) }
    } else {
        if (prec == 0) { OSANN_PREP_K(2, 0) }
        else { OSANN_PREP_K(2, 1) }
    }
#undef OSANN_PREP_K
#undef OSANN_PREP
    return count_launch();
}

int launch_tc_scan(int prec, const void* maps, const uint32_t* perm, const float4* rowstat, const void* Y16,
                   const float4* qstat, const float* tcs, const int64_t* query_src, int64_t grid_w, int radius,
                   const BatchedBuffers& b, uint32_t* Ubits, uint32_t* surv_cnt, uint32_t* surv, int cap,
                   uint32_t* status, unsigned long long* diag, const float* xs, const float* Y, int64_t S, int d,
                   int d_pad, int k, float cdot2, float Bn, float cabs, int debug, cudaStream_t st, int num_sms,
                   int layout)
{
    TcArgs a{};
    a.perm = perm;
    a.rowstat = rowstat;
    a.Y16 = static_cast<const uint16_t*>(Y16);
    a.qstat = qstat;
    a.tcs = tcs;
    a.query_src = query_src;
    a.items = b.items;
    a.n_items_dev = b.n_items_dev;
    a.qcount = b.qcount;
    a.qoff = b.qoff;
    a.qlist = b.qlist;
    a.counter = b.counters;
    a.Ubits = Ubits;
    a.surv_cnt = surv_cnt;
    a.surv = surv;
    a.status = status;
    a.diag = diag;
    a.xs = xs;
    a.Y = Y;
    a.S = S;
    a.grid_w = grid_w;
    a.d = d;
    a.d_pad = d_pad;
    a.k = k;
    a.radius = radius;
    a.cap = cap;
    a.stages = tc_stages(d_pad);
    a.abufs = tc_abufs(d_pad);
    if (a.stages > TC_STAGES_MAX || a.abufs > TC_NA_MAX) return -2;  // unsupported shape
    a.debug = debug;
    a.cdot2 = cdot2;
    a.Bn = Bn;
    a.cabs = cabs;
    const bool excl = query_src != nullptr;
    if (d_pad == 128 && !excl && layout != OSANN_LAYOUT_SMEM) {
        // one CTA per SM with the query tiles in TMEM and five cone-tile stages
        a.stages = tc_stages_at(d_pad);
        return launch_tc_scan_tmem(maps, a, k, prec, debug != 0, st, num_sms);
    }
    if (debug) return launch_tc_scan_debug(maps, a, k, prec, excl, st, num_sms);
#define OSANN_TC(KM)                                                                                 \
    do {                                                                                             \
        if (prec == 0)                                                                               \
            return excl ? launch_tc_t<KM, true, 0, false>(maps, a, st, num_sms)                      \
                        : launch_tc_t<KM, false, 0, false>(maps, a, st, num_sms);                    \
        return excl ? launch_tc_t<KM, true, 1, false>(maps, a, st, num_sms)                          \
                    : launch_tc_t<KM, false, 1, false>(maps, a, st, num_sms);                        \
    } while (0)
    if (k <= 1) OSANN_TC(1);
    if (k <= 4) OSANN_TC(4);
    if (k <= 16) OSANN_TC(16);
    OSANN_TC(32);
#undef OSANN_TC
}

int launch_tc_rerank(const float* xs, int d_pad, const uint32_t* perm, const uint32_t* offsets, uint32_t NC,
                     const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, const uint32_t* surv_cnt,
                     const uint32_t* surv, int cap, int k, const int64_t* query_src, int64_t grid_w, int radius,
                     unsigned long long* diag, uint32_t* ovf, int64_t* out_ids, float* out_d, cudaStream_t st)
{
    if (Q == 0) return 0;
    cudaMemsetAsync(ovf, 0, 4, st);
    const unsigned blocks = unsigned((Q * 32 + 127) / 128);
    const bool excl = query_src != nullptr;
#define OSANN_RR(F, KM)                                                                                           \
    do {                                                                                                          \
        if (excl)                                                                                                 \
            tc_rerank_kernel<F, KM, true><<<blocks, 128, 0, st>>>(xs, d_pad, perm, offsets, NC, Y, d, Q, probes,  \
                                                                  P_eff, surv_cnt, surv, cap, k, query_src,       \
                                                                  grid_w, radius, diag, ovf, out_ids, out_d);     \
        else                                                                                                      \
            tc_rerank_kernel<F, KM, false><<<blocks, 128, 0, st>>>(xs, d_pad, perm, offsets, NC, Y, d, Q, probes, \
                                                                   P_eff, surv_cnt, surv, cap, k, query_src,      \
                                                                   grid_w, radius, diag, ovf, out_ids, out_d);    \
    } while (0)
#define OSANN_RR_K(F)              \
    if (k <= 1) OSANN_RR(F, 1);    \
    else if (k <= 4) OSANN_RR(F, 4); \
    else if (k <= 16) OSANN_RR(F, 16); \
    else OSANN_RR(F, 32);
    if (d_pad <= 128) {
        OSANN_RR_K(1)
    } else {
        OSANN_RR_K(2)
    }
#undef OSANN_RR_K
#undef OSANN_RR
    return count_launch();
}

}  // namespace osann
