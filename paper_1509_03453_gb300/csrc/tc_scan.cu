// Batched candidate scan with bf16 tensor-core screening and an exact fp32
// rerank (the batched path's precision option).
//
// For a work item (cone c, group of up to 128 queries that probe it) the
// squared distances are first estimated on the 5th-generation tensor cores
// as  d~ = |q|^2 + |x|^2 - 2 q~.x~  (q~, x~ rounded to bf16, products exact,
// fp32 accumulation in TMEM), M = 128 queries x N = 128 cone rows per MMA
// group, the cone rows streamed by TMA (2-D tensor map over the bf16 copy of
// the permuted vectors, swizzled K-major tiles).  Each query keeps an upper
// bound U on its k-th best exact distance; a row survives the screen when
//     d~ - E(q, x) <= U,   E = 2 c |q| |x| + B (|q|^2 + |x|^2),
// where c bounds the bf16 rounding of both operands plus the fp32
// accumulation (c = 2u + u^2 + K 2^-22, u = 2^-8) and B the fp32 error of
// the norms plus a cushion for the fp32 rounding of the exact distance.  A
// discarded row is therefore provably farther than some candidate already
// seen, so the survivors contain the exact top-k.  Survivors are appended to
// a per-query list; the rerank computes their canonical fp32 distance (the
// same expression as every other path) and selects the top-k, so the result
// is bit-identical to the fp32 paths.  A query whose list overflows is
// rescanned in full by the rerank (counted).
#include <cuda.h>

#include "osann_device.cuh"
#include "osann_launch.h"
#include "osann_tc.cuh"

namespace osann {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;  // queries per item = MMA M
constexpr int TC_N = 128;  // cone rows per tile = MMA N = TMEM columns

__host__ __device__ inline int tc_row_bytes(int d_pad) { return d_pad >= 64 ? 128 : d_pad * 2; }
__host__ __device__ inline int tc_kblocks(int d_pad) { return d_pad >= 64 ? d_pad / 64 : 1; }
__host__ inline int tc_stages(int d_pad) { return d_pad <= 32 ? 4 : (d_pad == 64 ? 3 : 2); }

struct TcArgs {
    const uint32_t* offsets;
    const uint32_t* perm;
    const float4* rowstat;    // per row: ((1-B)|x|^2, |x|, |x|^2, 0); N + TC_N rows
    const __nv_bfloat16* Yb;  // Q x d_pad
    const float4* qstat;      // per query: (|q|^2, |q|, 0, 0)
    const int64_t* query_src;
    const uint2* items;
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
    int d, d_pad, k, radius, cap, stages, debug;
    float cdot2;  // 2c
    float Bn;     // B
};

template <int KMAX, bool EXCL>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_scan_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 const TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bfull[4];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ uint32_t item_sh;
    __shared__ int fail_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row_bytes = tc_row_bytes(a.d_pad);
    const int kblocks = tc_kblocks(a.d_pad);
    const int epb = row_bytes / 2;                 // bf16 elements per row block
    const int ksteps_pb = epb / 16;                // MMA K-steps per row block
    const int tileA = TC_M * a.d_pad * 2, tileB = TC_N * a.d_pad * 2;
    const int S = a.stages;
    unsigned char* sA = base;
    unsigned char* sB = base + tileA;
    float4* sR = reinterpret_cast<float4*>(sB + size_t(S) * tileB);
    const uint32_t n_items = *a.n_items_dev;
    const uint32_t idesc = idesc_bf16_f32(TC_M, TC_N);
    const uint32_t tx_bytes = uint32_t(tileB + TC_N * 16);

    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, TC_N);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bfull[s], 1);
        mbar_init(&mma_bar, 1);
        fence_mbar_init();
        fail_sh = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto issue_tile = [&](uint32_t g, int y0) {
        const int s = int(g % uint32_t(S));
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bfull[s], tx_bytes);
        for (int kb = 0; kb < kblocks; ++kb)
            tma_load_2d(sB + size_t(s) * tileB + size_t(kb) * TC_N * row_bytes, &tmap, kb * epb, y0, &bfull[s]);
        bulk_g2s(sR + size_t(s) * TC_N, a.rowstat + y0, TC_N * 16, &bfull[s]);
    };

    uint32_t gt = 0;      // tiles consumed by this CTA (stage ring position)
    uint32_t mphase = 0;  // parity of the next MMA completion
    bool failed = false;
    int pending_from = 0, pending_to = 0;  // issued-not-consumed tiles [from, to) of the current item

    for (;;) {
        if (tid == 0) item_sh = atomicAdd(a.counter, 1u);
        __syncthreads();
        const uint32_t item = item_sh;
        __syncthreads();
        if (item >= n_items) break;

        const uint2 bg = a.items[item];
        const uint32_t r0 = __ldg(a.offsets + bg.x), r1 = __ldg(a.offsets + bg.x + 1);
        const uint32_t cnt = a.qcount[bg.x];
        const uint32_t qbeg = a.qoff[bg.x] + bg.y * TC_M;
        const uint32_t qn = min(cnt - bg.y * TC_M, uint32_t(TC_M));
        const bool active = uint32_t(tid) < qn;
        int64_t slot = 0, q = 0;
        if (active) {
            slot = int64_t(a.qlist[qbeg + tid]);
            q = slot / a.S;
        }
        // this thread's query row of A, written in the swizzled K-major layout
        {
            const uint4* src = reinterpret_cast<const uint4*>(a.Yb + q * int64_t(a.d_pad));
            const int chunks = row_bytes / 16;
            for (int kb = 0; kb < kblocks; ++kb)
                for (int c = 0; c < chunks; ++c) {
                    uint4 v = active ? src[kb * chunks + c] : make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(sA + size_t(kb) * TC_M * row_bytes + swz_offset(tid, c, row_bytes)) = v;
                }
        }
        float qn2 = 0.f, qnorm = 0.f, U = INFINITY;
        if (active) {
            const float4 st = a.qstat[q];
            qn2 = st.x;
            qnorm = st.y;
            U = __uint_as_float(a.Ubits[q]);
        }
        const float Aq = a.cdot2 * qnorm;
        const float omb = 1.0f - a.Bn;
        float ubl[KMAX];  // k smallest upper bounds seen by this thread in this item (ascending)
#pragma unroll
        for (int j = 0; j < KMAX; ++j) ubl[j] = INFINITY;
        float Uthr = U - omb * qn2;  // survive iff (1-B)|x|^2 - A|x| - 2 acc <= Uthr
        int64_t src = EXCL && active ? a.query_src[q] : -1;

        fence_proxy_async_smem();
        __syncthreads();

        const int ntiles = int((r1 - r0 + TC_N - 1) / TC_N);
        if (tid == 0)
            for (int t = 0; t < ntiles && t < S; ++t) issue_tile(gt + uint32_t(t), int(r0) + t * TC_N);
        pending_from = 0;
        pending_to = ntiles < S ? ntiles : S;

        for (int t = 0; t < ntiles; ++t) {
            const uint32_t g = gt;
            const int s = int(g % uint32_t(S));
            if (tid == 0) {
                bool ok = mbar_wait_bounded(&bfull[s], (g / uint32_t(S)) & 1u);
                if (ok) {
                    tc_fence_after();
                    const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB + size_t(s) * tileB);
                    const int ksteps = kblocks * ksteps_pb;
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const int kb = kk / ksteps_pb, w = kk % ksteps_pb;
                        const uint32_t off_a = uint32_t(kb * TC_M * row_bytes + w * 32);
                        const uint32_t off_b = uint32_t(kb * TC_N * row_bytes + w * 32);
                        mma_bf16_ss(tmem, smem_desc_kmajor(aaddr + off_a, row_bytes),
                                    smem_desc_kmajor(baddr + off_b, row_bytes), idesc, kk > 0 ? 1u : 0u);
                    }
                    mma_commit(&mma_bar);
                } else {
                    fail_sh = 1;
                }
            }
            if (__syncthreads_or(tid == 0 && fail_sh)) {
                failed = true;
                pending_from = t;
                break;
            }
            const bool mok = mbar_wait_bounded(&mma_bar, mphase);
            mphase ^= 1u;
            if (__syncthreads_or(!mok)) {
                failed = true;
                pending_from = t + 1;
                break;
            }
            tc_fence_after();

            // ---- epilogue: screen the tile's columns for this thread's query
            const int y0 = int(r0) + t * TC_N;
            const int nvalid = min(TC_N, int(r1) - y0);
            const float4* srow = sR + size_t(s) * TC_N;
            const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
            for (int c0 = 0; c0 < nvalid; c0 += 32) {
                float acc[32];
                tmem_ld32(taddr + uint32_t(c0), acc);
                if (active) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float4 rs = srow[c0 + j];
                        float v = fmaf(-Aq, rs.y, rs.x);
                        v = fmaf(-2.0f, acc[j], v);
                        if (v <= Uthr && c0 + j < nvalid) {
                            const uint32_t row = uint32_t(y0 + c0 + j);
                            if (EXCL) {
                                const uint32_t id = __ldg(a.perm + row);
                                const int64_t dr = int64_t(id) / a.grid_w - src / a.grid_w;
                                const int64_t dc = int64_t(id) % a.grid_w - src % a.grid_w;
                                const int64_t adr = dr < 0 ? -dr : dr, adc = dc < 0 ? -dc : dc;
                                if (src >= 0 && (adr > adc ? adr : adc) <= a.radius) continue;
                            }
                            const uint32_t pos = atomicAdd(a.surv_cnt + q, 1u);
                            if (pos < uint32_t(a.cap)) a.surv[q * a.cap + pos] = row;
                            // upper bound on this row's exact distance
                            const float dt = fmaf(-2.0f, acc[j], qn2 + rs.z);
                            const float ub = fmaxf(dt + fmaf(Aq, rs.y, a.Bn * (qn2 + rs.z)), 0.0f);
                            if (ub < ubl[KMAX - 1]) {
#pragma unroll
                                for (int u = KMAX - 1; u > 0; --u) {
                                    const float pu = ubl[u - 1];
                                    if (pu > ub) ubl[u] = pu;
                                    else if (ubl[u] > ub) ubl[u] = ub;
                                }
                                if (ubl[0] > ub) ubl[0] = ub;
                            }
                            // the k-th smallest bound of k distinct candidates bounds the k-th best
                            float kth = INFINITY;
#pragma unroll
                            for (int u = 0; u < KMAX; ++u)
                                if (u == a.k - 1) kth = ubl[u];
                            if (kth < U) {
                                U = kth;
                                Uthr = U - omb * qn2;
                            }
                        }
                    }
                    if (a.debug && lane < nvalid - c0) {
                        // tensor-core dot product against an fp32 one for one column per thread
                        const float* xr = a.xs + size_t(y0 + c0 + lane) * a.d_pad;
                        const float* yr = a.Y + q * int64_t(a.d);
                        float dot = 0.f;
                        for (int i = 0; i < a.d; ++i) dot = fmaf(xr[i], yr[i], dot);
                        float accl = 0.f;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j == lane) accl = acc[j];
                        const float lim = 0.5f * a.cdot2 * qnorm * srow[c0 + lane].y * 1.0001f +
                                          1e-6f * (qn2 + srow[c0 + lane].z) + 1e-30f;
                        atomicAdd(a.diag + 2, 1ull);
                        if (fabsf(accl - dot) > lim) {
                            atomicAdd(a.diag + 3, 1ull);
                            atomicOr(a.status, ST_BOUND);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            ++gt;
            if (tid == 0 && t + S < ntiles) issue_tile(gt + uint32_t(S - 1), int(r0) + (t + S) * TC_N);
            pending_from = t + 1;
            pending_to = ntiles < t + 1 + S ? ntiles : t + 1 + S;
        }
        if (failed) break;
        if (active) atomicMin(a.Ubits + q, __float_as_uint(fmaxf(U, 0.0f)));
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(a.status, ST_TIMEOUT);
            // let tiles still in flight land before shared memory goes away
            for (int t = pending_from; t < pending_to; ++t) {
                const uint32_t g = gt + uint32_t(t - pending_from);
                mbar_wait_bounded(&bfull[g % uint32_t(S)], (g / uint32_t(S)) & 1u);
            }
            mbar_wait_bounded(&mma_bar, mphase);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_N);
}

// ---------------------------------------------------------------- query prep

// One warp per query: bf16 copy, norms, survivor counter reset, and the
// initial upper bound U: k rows of the first probed cone holding at least k
// rows (their fp32 distances, inflated by the fp32 error bound), or +inf.
__global__ void __launch_bounds__(128) tc_query_prep_kernel(const float* __restrict__ Y, int64_t Q, int d, int d_pad,
                                                            const uint32_t* __restrict__ probes, int64_t P_eff,
                                                            const uint32_t* __restrict__ offsets, uint32_t NC,
                                                            const float* __restrict__ xs, int k, int seed,
                                                            __nv_bfloat16* __restrict__ Yb, float4* __restrict__ qstat,
                                                            uint32_t* __restrict__ Ubits,
                                                            uint32_t* __restrict__ surv_cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const float* y = Y + q * int64_t(d);
    float s = 0.f;
    for (int c = lane * 4; c < d_pad; c += 128) {
        float4 v;
        v.x = c + 0 < d ? y[c + 0] : 0.f;
        v.y = c + 1 < d ? y[c + 1] : 0.f;
        v.z = c + 2 < d ? y[c + 2] : 0.f;
        v.w = c + 3 < d ? y[c + 3] : 0.f;
        __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(Yb + q * int64_t(d_pad) + c) = pk;
        s = fmaf(v.x, v.x, s);
        s = fmaf(v.y, v.y, s);
        s = fmaf(v.z, v.z, s);
        s = fmaf(v.w, v.w, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    float U = INFINITY;
    if (seed) {
        for (int64_t p = 0; p < P_eff; ++p) {
            const uint32_t b = probes[q * P_eff + p];
            if (b >= NC) continue;
            const uint32_t o0 = offsets[b], o1 = offsets[b + 1];
            if (o1 - o0 < uint32_t(k)) continue;
            float worst = 0.f;
            for (int j = 0; j < k; ++j) {
                const float* xr = xs + size_t(o0 + j) * d_pad;
                float t = 0.f;
                for (int c = lane; c < d; c += 32) {
                    const float df = xr[c] - y[c];
                    t = fmaf(df, df, t);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                worst = fmaxf(worst, t);
            }
            // any summation order is within (d + 6) 2^-24 relative of the exact value
            U = worst * (1.0f + float(d + 8) * 5.9604645e-8f) + 1e-30f;
            break;
        }
    }
    if (lane == 0) {
        qstat[q] = make_float4(s, sqrtf(s), 0.f, 0.f);
        Ubits[q] = __float_as_uint(U);
        surv_cnt[q] = 0;
    }
}

// ---------------------------------------------------------------- rerank

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
                                                        int64_t* __restrict__ out_ids, float* __restrict__ out_d)
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
    auto consider = [&](uint32_t row, bool valid) {
        const float4* xr = reinterpret_cast<const float4*>(xs + size_t(valid ? row : 0) * d_pad) + sub * F;
        float cpart[F];
#pragma unroll
        for (int f = 0; f < F; ++f) cpart[f] = sq4(xr[f], qv[f]);
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
        for (uint32_t b0 = 0; b0 < n; b0 += CPP) {
            const uint32_t i = b0 + g;
            const bool valid = i < n;
            consider(valid ? surv[q * cap + i] : 0u, valid);
        }
        if (lane == 0) atomicAdd(diag, (unsigned long long)n);
    } else {
        if (lane == 0) atomicAdd(diag + 1, 1ull);
        for (int64_t p = 0; p < P_eff; ++p) {
            const uint32_t b = probes[q * P_eff + p];
            if (b >= NC) continue;
            const uint32_t o0 = offsets[b], o1 = offsets[b + 1];
            for (uint32_t b0 = o0; b0 < o1; b0 += CPP) {
                const uint32_t r = b0 + g;
                consider(r, r < o1);
            }
        }
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

int tc_encode_rows_map(void* map_out, const __nv_bfloat16* xb, int64_t N, int d_pad)
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
    const int row_bytes = tc_row_bytes(d_pad);
    const cuuint64_t dims[2] = {cuuint64_t(d_pad), cuuint64_t(N)};
    const cuuint64_t strides[1] = {cuuint64_t(d_pad) * 2};
    const cuuint32_t box[2] = {cuuint32_t(row_bytes / 2), cuuint32_t(TC_N)};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                   : (row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                      : CU_TENSOR_MAP_SWIZZLE_32B);
    CUresult r = fn(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<__nv_bfloat16*>(xb), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", int(r));
        return -5;
    }
    return 0;
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

int launch_tc_query_prep(const float* Y, int64_t Q, int d, int d_pad, const uint32_t* probes, int64_t P_eff,
                         const uint32_t* offsets, uint32_t NC, const float* xs, int k, bool seed, __nv_bfloat16* Yb,
                         float4* qstat, uint32_t* Ubits, uint32_t* surv_cnt, cudaStream_t st)
{
    if (Q == 0) return 0;
    tc_query_prep_kernel<<<unsigned((Q * 32 + 127) / 128), 128, 0, st>>>(Y, Q, d, d_pad, probes, P_eff, offsets, NC,
                                                                         xs, k, seed ? 1 : 0, Yb, qstat, Ubits,
                                                                         surv_cnt);
    return count_launch();
}

size_t tc_smem_bytes(int d_pad)
{
    const size_t need = 1024 + size_t(TC_M) * d_pad * 2 + size_t(tc_stages(d_pad)) * (size_t(TC_N) * d_pad * 2 + TC_N * 16);
    // at least 47 KB so that at most four CTAs (4 x 128 TMEM columns) share an SM
    return need < 47u * 1024u ? 47u * 1024u : need;
}

template <int KMAX, bool EXCL>
static int launch_tc_t(const void* map, const TcArgs& a, cudaStream_t st, int num_sms)
{
    const size_t smem = tc_smem_bytes(a.d_pad);
    auto kern = tc_scan_kernel<KMAX, EXCL>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TC_THREADS, smem);
    if (occ < 1) occ = 1;
    if (occ > 4) occ = 4;
    kern<<<unsigned(num_sms * occ), TC_THREADS, smem, st>>>(*static_cast<const CUtensorMap*>(map), a);
    return count_launch();
}

int launch_tc_scan(const void* map, const uint32_t* offsets, const uint32_t* perm, const float4* rowstat,
                   const __nv_bfloat16* Yb, const float4* qstat, const int64_t* query_src, int64_t grid_w, int radius,
                   const BatchedBuffers& b, uint32_t* Ubits, uint32_t* surv_cnt, uint32_t* surv, int cap,
                   uint32_t* status, unsigned long long* diag, const float* xs, const float* Y, int64_t S, int d,
                   int d_pad, int k, float cdot2, float Bn, int debug, cudaStream_t st, int num_sms)
{
    TcArgs a{};
    a.offsets = offsets;
    a.perm = perm;
    a.rowstat = rowstat;
    a.Yb = Yb;
    a.qstat = qstat;
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
    a.debug = debug;
    a.cdot2 = cdot2;
    a.Bn = Bn;
    const bool excl = query_src != nullptr;
#define OSANN_TC(KM)                                                                                     \
    return excl ? launch_tc_t<KM, true>(map, a, st, num_sms) : launch_tc_t<KM, false>(map, a, st, num_sms)
    if (k <= 1) OSANN_TC(1);
    if (k <= 4) OSANN_TC(4);
    if (k <= 16) OSANN_TC(16);
    OSANN_TC(32);
#undef OSANN_TC
}

int launch_tc_rerank(const float* xs, int d_pad, const uint32_t* perm, const uint32_t* offsets, uint32_t NC,
                     const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, const uint32_t* surv_cnt,
                     const uint32_t* surv, int cap, int k, const int64_t* query_src, int64_t grid_w, int radius,
                     unsigned long long* diag, int64_t* out_ids, float* out_d, cudaStream_t st)
{
    if (Q == 0) return 0;
    const unsigned blocks = unsigned((Q * 32 + 127) / 128);
    const bool excl = query_src != nullptr;
#define OSANN_RR(F, KM)                                                                                           \
    do {                                                                                                          \
        if (excl)                                                                                                 \
            tc_rerank_kernel<F, KM, true><<<blocks, 128, 0, st>>>(xs, d_pad, perm, offsets, NC, Y, d, Q, probes,  \
                                                                  P_eff, surv_cnt, surv, cap, k, query_src,       \
                                                                  grid_w, radius, diag, out_ids, out_d);          \
        else                                                                                                      \
            tc_rerank_kernel<F, KM, false><<<blocks, 128, 0, st>>>(xs, d_pad, perm, offsets, NC, Y, d, Q, probes, \
                                                                   P_eff, surv_cnt, surv, cap, k, query_src,      \
                                                                   grid_w, radius, diag, out_ids, out_d);         \
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
