// Plain per-query candidate scan (Algorithm 1 with one basis): for each
// query, visit its probed cones in order and compute the exact squared
// Euclidean distance (Eq. 1) to every point of every visited cone, keeping
// the k nearest by (distance, id).  Distances are fp32 direct differences.
//
// One CTA per query (or, with a device query list, a grid-stride loop over
// the listed queries with the stage ring's phases carried across them).
// Thread 0 streams the rows of the visited cones from
// the permuted vector array into a ring of shared-memory stages with 1-D
// bulk copies (TMA engine), each stage guarded by an mbarrier.  The CTA
// consumes a stage with TPR = min(32, d_pad/4) adjacent threads per row,
// each holding one or two float4 pieces of the query: a quarter-warp reads
// 128 contiguous bytes (no bank conflicts) and the row's distance is the
// canonical piece tree of osann_device.cuh, finished with shuffles.  The
// row's leading thread keeps a register top-k; the CTA merges the
// per-thread lists at the end.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

constexpr int PLAIN_THREADS = 128;
constexpr int PLAIN_STAGES = 4;
constexpr int PLAIN_STAGE_FLOATS = 4096;  // 16 KB per stage

__device__ __forceinline__ bool excluded_pair(uint32_t id, int64_t src, int64_t grid_w, int radius)
{
    if (src < 0) return false;
    int64_t dr = int64_t(id) / grid_w - src / grid_w;
    int64_t dc = int64_t(id) % grid_w - src % grid_w;
    dr = dr < 0 ? -dr : dr;
    dc = dc < 0 ? -dc : dc;
    return (dr > dc ? dr : dc) <= radius;
}

template <int KMAX>
__device__ __forceinline__ void block_merge_write(uint64_t (&list)[KMAX], int k, int64_t* out_ids, float* out_d,
                                                  uint64_t* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < k; ++j) {
        const uint64_t head = topk_head<KMAX>(list, k);
        uint64_t m = warp_min_u64(head);
        if (lane == 0) red[warp] = m;
        __syncthreads();
        uint64_t best = red[0];
#pragma unroll
        for (int w = 1; w < PLAIN_THREADS / 32; ++w) best = red[w] < best ? red[w] : best;
        if (head == best && best != EMPTY_DI) topk_remove<KMAX>(list, k, best);
        if (threadIdx.x == 0) {
            const uint32_t id = di_id(best);
            out_ids[j] = id == 0xFFFFFFFFu ? int64_t(-1) : int64_t(id);
            out_d[j] = di_dist(best);
        }
        __syncthreads();
    }
}

template <int F, int KMAX, bool EXCL>
__global__ void __launch_bounds__(PLAIN_THREADS) plain_scan_kernel(
    const float* __restrict__ xs, const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ perm, int d_pad,
    const float* __restrict__ Y, int d, const uint32_t* __restrict__ probes, int64_t P_eff, uint32_t NC, int k,
    const int64_t* __restrict__ query_src, int64_t grid_w, int radius, const uint32_t* __restrict__ qlist,
    int64_t Q, int64_t* __restrict__ out_ids, float* __restrict__ out_d, uint32_t* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage_buf = reinterpret_cast<float*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[PLAIN_STAGES];
    __shared__ int2 meta[PLAIN_STAGES];  // (first row, row count or -1 = no chunk)
    __shared__ uint64_t red[PLAIN_THREADS / 32];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int n4 = d_pad >> 2;               // float4 pieces per row
    const int TPR = n4 / F;                  // threads per row (<= 32)
    const int RPP = PLAIN_THREADS / TPR;     // rows per pass
    const int RPC = PLAIN_STAGE_FLOATS / d_pad;  // rows per chunk (a multiple of RPP)
    const int r_in = tid / TPR, sub = tid % TPR;

    if (tid == 0) {
        for (int s = 0; s < PLAIN_STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    // qlist: [count, q_0, q_1, ...] (count <= Q); null: queries 0..Q-1
    int64_t nq = Q;
    if (qlist) nq = qlist[0] < uint64_t(Q) ? int64_t(qlist[0]) : Q;
    int c = 0;  // chunk counter, carried across queries: stage c % S, phase (c / S) & 1
    for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int64_t q = qlist ? int64_t(qlist[1 + qi]) : qi;
        const int64_t src = EXCL ? query_src[q] : -1;

        // pieces sub*F .. sub*F+F-1 of the query
        float4 qv[F];
        {
            const float* y = Y + q * int64_t(d);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const int cc = 4 * (sub * F + f);
                qv[f].x = cc + 0 < d ? y[cc + 0] : 0.0f;
                qv[f].y = cc + 1 < d ? y[cc + 1] : 0.0f;
                qv[f].z = cc + 2 < d ? y[cc + 2] : 0.0f;
                qv[f].w = cc + 3 < d ? y[cc + 3] : 0.0f;
            }
        }
        uint64_t list[KMAX];
        topk_init<KMAX>(list, k);

        // producer state (thread 0 only)
        int64_t pi = 0;
        uint32_t cur = 0, cur_end = 0;
        const uint32_t* qprobes = probes + q * P_eff;
        auto issue = [&](int s) {
            while (cur >= cur_end && pi < P_eff) {
                const uint32_t b = qprobes[pi++];
                if (b >= NC) continue;  // never produced by the probe kernel; guards the offsets read
                cur = offsets[b];
                cur_end = offsets[b + 1];
            }
            if (cur >= cur_end) {
                meta[s] = make_int2(0, -1);
                return;
            }
            const uint32_t n = cur_end - cur < uint32_t(RPC) ? cur_end - cur : uint32_t(RPC);
            meta[s] = make_int2(int(cur), int(n));
            const uint32_t bytes = n * uint32_t(d_pad) * 4u;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[s], bytes);
            bulk_g2s(stage_buf + size_t(s) * PLAIN_STAGE_FLOATS, xs + size_t(cur) * d_pad, bytes, &bars[s]);
            cur += n;
        };

        // no copy is in flight here: the previous query ended on S empty stages
        if (tid == 0)
            for (int i = 0; i < PLAIN_STAGES; ++i) issue((c + i) % PLAIN_STAGES);
        __syncthreads();

        for (;; ++c) {
            const int s = c % PLAIN_STAGES;
            const int2 m = meta[s];
            if (m.y < 0) break;
            const bool ok = mbar_wait_bounded(&bars[s], uint32_t((c / PLAIN_STAGES) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(status, ST_TIMEOUT);
                    abort_flag = 1;
                }
                break;
            }
            const float* stage = stage_buf + size_t(s) * PLAIN_STAGE_FLOATS;
            for (int r0 = 0; r0 < m.y; r0 += RPP) {
                // rows past the chunk's end (still inside the stage) read stale
                // memory; their result is discarded
                const int r = r0 + r_in;
                const float4* row = reinterpret_cast<const float4*>(stage + size_t(r) * d_pad) + sub * F;
                float cpart[F];
#pragma unroll
                for (int f = 0; f < F; ++f) cpart[f] = sq4(row[f], qv[f]);
                const float dist = lane_tree(pair_tree<F>(cpart), TPR);
                if (sub == 0 && r < m.y) {
                    const uint32_t rowid = uint32_t(m.x + r);
                    if (EXCL) {
                        const uint32_t id = __ldg(perm + rowid);
                        if (!excluded_pair(id, src, grid_w, radius)) {
                            const uint64_t v = pack_di(dist, id);
                            if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                        }
                    } else if (dist <= di_dist(list[KMAX - 1])) {
                        const uint64_t v = pack_di(dist, __ldg(perm + rowid));
                        if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                    }
                }
            }
            __syncthreads();
            if (tid == 0) issue(s);
        }
        if (abort_flag) {
            // let copies still in flight land before the CTA's shared memory goes away
            if (tid == 0)
                for (int i = 0; i < PLAIN_STAGES; ++i) {
                    const int cc = c + i, ss = cc % PLAIN_STAGES;
                    if (meta[ss].y >= 0) mbar_wait_bounded(&bars[ss], uint32_t((cc / PLAIN_STAGES) & 1));
                }
            __syncthreads();
            block_merge_write<KMAX>(list, k, out_ids + q * k, out_d + q * k, red);
            return;
        }
        block_merge_write<KMAX>(list, k, out_ids + q * k, out_d + q * k, red);
    }
}

template <int F, int KMAX, bool EXCL>
static int launch_plain_t(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad, const float* Y,
                          int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC, int k,
                          const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist,
                          int64_t grid, int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st)
{
    const int smem = PLAIN_STAGES * PLAIN_STAGE_FLOATS * 4;
    auto kern = plain_scan_kernel<F, KMAX, EXCL>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    kern<<<unsigned(grid), PLAIN_THREADS, smem, st>>>(xs, offsets, perm, d_pad, Y, d, probes, P_eff, NC, k,
                                                      query_src, grid_w, radius, qlist, Q, out_ids, out_d, status);
    return count_launch();
}

template <int F, bool EXCL>
static int launch_plain_k(int k, const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad,
                          const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC,
                          const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist, int64_t grid,
                          int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st)
{
#define OSANN_PLAIN(KM)                                                                                      \
    return launch_plain_t<F, KM, EXCL>(xs, offsets, perm, d_pad, Y, d, Q, probes, P_eff, NC, k, query_src, grid_w, \
                                       radius, qlist, grid, out_ids, out_d, status, st)
    if (k <= 1) OSANN_PLAIN(1);
    if (k <= 4) OSANN_PLAIN(4);
    if (k <= 16) OSANN_PLAIN(16);
    OSANN_PLAIN(32);
#undef OSANN_PLAIN
}

int launch_plain_scan(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad, const float* Y,
                      int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC, int k,
                      const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist, int num_sms,
                      int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st)
{
    if (Q == 0) return 0;
    const bool excl = query_src != nullptr;
    // a listed subset of unknown size: a grid-stride loop over three CTAs per SM
    int64_t grid = Q;
    if (qlist) {
        const int64_t g = int64_t(num_sms) * 3;
        grid = Q < g ? Q : g;
    }
#define OSANN_PLAIN_F(F, EX)                                                                                     \
    return launch_plain_k<F, EX>(k, xs, offsets, perm, d_pad, Y, d, Q, probes, P_eff, NC, query_src, grid_w, radius, \
                                 qlist, grid, out_ids, out_d, status, st)
    // d_pad in {16, 32, 64, 128}: one piece per thread; 256: two
    if (d_pad <= 128) {
        if (excl) OSANN_PLAIN_F(1, true);
        OSANN_PLAIN_F(1, false);
    }
    if (excl) OSANN_PLAIN_F(2, true);
    OSANN_PLAIN_F(2, false);
#undef OSANN_PLAIN_F
}

}  // namespace osann
