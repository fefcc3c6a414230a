// Plain per-query candidate scan (Algorithm 1 with one basis): for each
// query, visit its probed cones in order and compute the exact squared
// Euclidean distance (Eq. 1) to every point of every visited cone, keeping
// the k nearest by (distance, id).  Distances are fp32 direct differences.
//
// A persistent grid of CTAs walks the queries (or a device list of them),
// each query's probe list in chunks of PLAIN_CHUNK cones.  Warp roles:
//   - one producer warp builds, for each chunk, a cone table in shared
//     memory (its lanes load the probes and offsets in parallel; a warp scan
//     turns the cone sizes into flat row positions, so the chunk's rows form
//     one sequence), then streams that sequence through a ring of 16 KB
//     stages, each stage filled with one 1-D bulk copy (TMA engine) per cone
//     segment it covers, the lanes issuing copies in parallel -- small cones
//     are packed into full stages and no copy waits on a global load;
//   - eight consumer warps compute the distances of each stage's rows with
//     TPR = min(32, d_pad/4) adjacent threads per row, each holding one or
//     two float4 pieces of the query (the canonical piece tree of
//     osann_device.cuh, finished with shuffles).  A row's leading thread
//     keeps a register top-k and maps a candidate's flat position back to
//     its point id (binary search in the chunk's table, then perm) only when
//     it enters the top-k (every row when an exclusion filter needs the id).
// Hand-offs are mbarriers -- stage full (an arrival per producer lane, plus
// the bulk copies' transaction bytes) / empty (one arrival per consumer warp), cone table full / empty (two tables, so the
// next chunk's table is built while the current one is consumed) -- so no
// block-wide barrier stands in the streaming loop; the consumers meet at a
// named barrier only when a query ends, to merge their lists.  Every wait is
// bounded; a wait that runs out sets ST_TIMEOUT and every role drops out
// after letting its copies in flight land.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

constexpr int PLAIN_CONSUMERS = 256;             // eight consumer warps
constexpr int PLAIN_THREADS = PLAIN_CONSUMERS + 32;  // plus the producer warp
constexpr int PLAIN_STAGES = 4;
constexpr int PLAIN_STAGE_FLOATS = 4096;  // 16 KB per stage
constexpr int PLAIN_CHUNK = 256;          // cones per table
constexpr int PLAIN_BAR = 1;              // named barrier of the consumer warps

// Clock budget of the stage waits (a test can shorten it through
// osann_debug_wait_budget to make the waits run out; the drain of copies
// still in flight after a timeout always uses the full budget).
static long long g_plain_wait_budget = WAIT_BUDGET_CYCLES;

void set_plain_wait_budget(long long cycles) { g_plain_wait_budget = cycles > 0 ? cycles : WAIT_BUDGET_CYCLES; }

__device__ __forceinline__ bool excluded_pair(uint32_t id, int64_t src, int64_t grid_w, int radius)
{
    if (src < 0) return false;
    int64_t dr = int64_t(id) / grid_w - src / grid_w;
    int64_t dc = int64_t(id) % grid_w - src % grid_w;
    dr = dr < 0 ? -dr : dr;
    dc = dc < 0 ? -dc : dc;
    return (dr > dc ? dr : dc) <= radius;
}

// Cone of flat row t of a chunk table: the last c with pre[c] <= t (empty
// cones share their prefix with the next one and are passed over).
// Requires pre[0] <= t < pre[PLAIN_CHUNK].
__device__ __forceinline__ int table_cone(const uint32_t* pre, uint32_t t)
{
    int lo = 0, hi = PLAIN_CHUNK;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Barrier of the consumer warps only (the producer warp never joins).
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync %0, %1;" ::"n"(PLAIN_BAR), "n"(PLAIN_CONSUMERS) : "memory");
}
// The same barrier, returning whether any consumer thread passed `pred`.
__device__ __forceinline__ bool consumers_sync_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "n"(PLAIN_BAR), "n"(PLAIN_CONSUMERS)
        : "memory");
    return r != 0;
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
        consumers_sync();
        uint64_t best = red[0];
#pragma unroll
        for (int w = 1; w < PLAIN_CONSUMERS / 32; ++w) best = red[w] < best ? red[w] : best;
        if (head == best && best != EMPTY_DI) topk_remove<KMAX>(list, k, best);
        if (threadIdx.x == 0) {
            const uint32_t id = di_id(best);
            out_ids[j] = id == 0xFFFFFFFFu ? int64_t(-1) : int64_t(id);
            out_d[j] = di_dist(best);
        }
        consumers_sync();
    }
}

// a chunk of a query's probe list, published by the producer with its table
struct PlainChunk {
    int64_t qi;      // query slot (-1: no more work)
    uint32_t total;  // rows of the chunk
    int first, last; // first / last chunk of its query
};

template <int F, int KMAX, bool EXCL>
__global__ void __launch_bounds__(PLAIN_THREADS) plain_scan_kernel(
    const float* __restrict__ xs, const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ perm, int d_pad,
    const float* __restrict__ Y, int d, const uint32_t* __restrict__ probes, int64_t P_eff, uint32_t NC, int k,
    const int64_t* __restrict__ query_src, int64_t grid_w, int radius, const uint32_t* __restrict__ qlist,
    int64_t Q, int64_t* __restrict__ out_ids, float* __restrict__ out_d, uint32_t* __restrict__ status,
    long long wait_budget)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage_buf = reinterpret_cast<float*>(smem_raw);
    __shared__ __align__(8) uint64_t full[PLAIN_STAGES], empty[PLAIN_STAGES], tfull[2], tempty[2];
    __shared__ uint32_t cpre[2][PLAIN_CHUNK + 1];  // flat row where each cone starts; [CHUNK] = total
    __shared__ uint32_t cstart[2][PLAIN_CHUNK];    // first row of each cone in xs
    __shared__ PlainChunk desc[2];
    __shared__ uint64_t red[PLAIN_CONSUMERS / 32];
    __shared__ volatile int abort_sh;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t row_bytes = uint32_t(d_pad) * 4u;
    const uint32_t RPC = uint32_t(PLAIN_STAGE_FLOATS / d_pad);  // rows per stage
    const int64_t nchunk = (P_eff + PLAIN_CHUNK - 1) / PLAIN_CHUNK;

    if (tid == 0) {
        for (int s = 0; s < PLAIN_STAGES; ++s) {
            mbar_init(&full[s], 32);  // one arrival per producer lane
            mbar_init(&empty[s], PLAIN_CONSUMERS / 32);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], PLAIN_CONSUMERS / 32);
        }
        fence_mbar_init();
        abort_sh = 0;
    }
    __syncthreads();

    // qlist: [count, q_0, q_1, ...] (count <= Q); null: queries 0..Q-1
    int64_t nq = Q;
    if (qlist) nq = qlist[0] < uint64_t(Q) ? int64_t(qlist[0]) : Q;
    auto query_of = [=](int64_t qi) -> int64_t { return qlist ? int64_t(qlist[1 + qi]) : qi; };
    // a wait that gives up when another role has dropped out, or its budget
    // runs out (a shortened budget skips the first try_wait, which may suspend
    // the thread until the phase completes)
    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (wait_budget >= WAIT_BUDGET_CYCLES && mbar_try_wait(bar, parity)) return true;
        if (abort_sh) return false;
        if (mbar_wait_bounded(bar, parity, wait_budget)) return true;
        atomicOr(status, ST_TIMEOUT);
        abort_sh = 1;
        return false;
    };

    if (warp == PLAIN_CONSUMERS / 32) {
        // ------------------------------------------------ producer warp
        uint32_t sc = 0;  // stages issued: slot sc % S, phase (sc / S) & 1
        uint32_t tc = 0;  // tables published: buffer tc & 1
        bool ok = true;
        for (int64_t qi = blockIdx.x; ok; qi += gridDim.x) {
            for (int64_t j = 0; j < (qi < nq ? nchunk : 1) && ok; ++j, ++tc) {
                const int b = int(tc & 1u);
                if (tc >= 2 && !wait(&tempty[b], ((tc >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                uint32_t total = 0;
                if (qi < nq) {
                    // eight cones per lane: sizes, lane-local prefix, warp scan of the lane totals
                    const int64_t q = query_of(qi);
                    uint32_t st[8], sz[8], run = 0;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int64_t p = j * PLAIN_CHUNK + lane * 8 + t;
                        st[t] = 0;
                        sz[t] = 0;
                        if (p < P_eff) {
                            const uint32_t cb = __ldg(probes + q * P_eff + p);
                            if (cb < NC) {  // never produced by the probe kernel; guards the offsets read
                                st[t] = __ldg(offsets + cb);
                                sz[t] = __ldg(offsets + cb + 1) - st[t];
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) run += sz[t];
                    uint32_t incl = run;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    total = __shfl_sync(0xffffffffu, incl, 31);
                    uint32_t pos = incl - run;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        cpre[b][lane * 8 + t] = pos;
                        cstart[b][lane * 8 + t] = st[t];
                        pos += sz[t];
                    }
                    if (lane == 0) cpre[b][PLAIN_CHUNK] = total;
                }
                if (lane == 0) {
                    PlainChunk c;
                    c.qi = qi < nq ? qi : -1;
                    c.total = total;
                    c.first = j == 0;
                    c.last = j == nchunk - 1;
                    desc[b] = c;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&tfull[b]);  // release: the table and descriptor are visible
                if (qi >= nq) {
                    ok = false;  // the end marker is out
                    break;
                }
                // stream the chunk's rows, cone cursor cc
                int cc = 0;
                const uint32_t nst = (total + RPC - 1) / RPC;
                for (uint32_t i = 0; i < nst; ++i, ++sc) {
                    const int s = int(sc % PLAIN_STAGES);
                    if (sc >= PLAIN_STAGES && !wait(&empty[s], ((sc / PLAIN_STAGES) - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    const uint32_t a = i * RPC, e = a + (total - a < RPC ? total - a : RPC);
                    if (lane == 0) mbar_arrive_expect_tx(&full[s], (e - a) * row_bytes);
                    else mbar_arrive(&full[s]);
                    fence_proxy_async_smem();
                    float* dst = stage_buf + size_t(s) * PLAIN_STAGE_FLOATS;
                    for (int base = cc;; base += 32) {
                        const int c = base + lane;
                        bool past = true;  // cone c ends at or after e (or is beyond the table)
                        if (c < PLAIN_CHUNK) {
                            const uint32_t p0 = cpre[b][c], p1 = cpre[b][c + 1];
                            const uint32_t s0 = p0 > a ? p0 : a, s1 = p1 < e ? p1 : e;
                            if (s1 > s0)
                                bulk_g2s(dst + size_t(s0 - a) * d_pad,
                                         xs + (size_t(cstart[b][c]) + (s0 - p0)) * d_pad, (s1 - s0) * row_bytes,
                                         &full[s]);
                            past = p1 > e;
                        }
                        const uint32_t m = __ballot_sync(0xffffffffu, past);
                        if (m) {
                            // the next stage starts in the first cone that reaches past e
                            cc = base + __ffs(int(m)) - 1;
                            break;
                        }
                    }
                }
            }
        }
        // let the copies still in flight land before shared memory goes away
        if (lane == 0 && abort_sh)
            for (uint32_t g = sc > uint32_t(PLAIN_STAGES) ? sc - uint32_t(PLAIN_STAGES) : 0u; g < sc; ++g)
                mbar_wait_bounded(&full[g % PLAIN_STAGES], (g / PLAIN_STAGES) & 1u);
    } else {
        // ------------------------------------------------ consumer warps
        const int n4 = d_pad >> 2;                // float4 pieces per row
        const int TPR = n4 / F;                   // threads per row (<= 32)
        const int RPP = PLAIN_CONSUMERS / TPR;    // rows per pass
        const int r_in = tid / TPR, sub = tid % TPR;
        uint64_t list[KMAX];
        float4 qv[F];
        int64_t q = 0, src = -1, done_q = blockIdx.x;  // queries before done_q are written
        uint32_t sc = 0;
        bool failed = false;
        for (uint32_t tc = 0;; ++tc) {
            const int b = int(tc & 1u);
            failed = !wait(&tfull[b], (tc >> 1) & 1u);
            const PlainChunk c = desc[b];
            if (consumers_sync_or(failed)) break;
            if (c.qi < 0) break;
            if (c.first) {
                q = query_of(c.qi);
                src = EXCL ? query_src[q] : -1;
                const float* y = Y + q * int64_t(d);
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    const int cc = 4 * (sub * F + f);
                    qv[f].x = cc + 0 < d ? y[cc + 0] : 0.0f;
                    qv[f].y = cc + 1 < d ? y[cc + 1] : 0.0f;
                    qv[f].z = cc + 2 < d ? y[cc + 2] : 0.0f;
                    qv[f].w = cc + 3 < d ? y[cc + 3] : 0.0f;
                }
                topk_init<KMAX>(list, k);
            }
            const uint32_t nst = (c.total + RPC - 1) / RPC;
            for (uint32_t i = 0; i < nst; ++i, ++sc) {
                const int s = int(sc % PLAIN_STAGES);
                if (!wait(&full[s], (sc / PLAIN_STAGES) & 1u)) {
                    failed = true;
                    break;
                }
                const uint32_t a = i * RPC;
                const int n = int(c.total - a < RPC ? c.total - a : RPC);
                const float* stage = stage_buf + size_t(s) * PLAIN_STAGE_FLOATS;
                for (int r0 = 0; r0 < n; r0 += RPP) {
                    // rows past the stage's fill (still inside the stage) read stale
                    // memory; their result is discarded
                    const int r = r0 + r_in;
                    const float4* row = reinterpret_cast<const float4*>(stage + size_t(r) * d_pad) + sub * F;
                    float cpart[F];
#pragma unroll
                    for (int f = 0; f < F; ++f) cpart[f] = sq4(row[f], qv[f]);
                    const float dist = lane_tree(pair_tree<F>(cpart), TPR);
                    if (sub == 0 && r < n && (EXCL || dist <= di_dist(list[KMAX - 1]))) {
                        const uint32_t t = a + uint32_t(r);
                        const int cn = table_cone(cpre[b], t);
                        const uint32_t id = __ldg(perm + cstart[b][cn] + (t - cpre[b][cn]));
                        if (!EXCL || !excluded_pair(id, src, grid_w, radius)) {
                            const uint64_t v = pack_di(dist, id);
                            if (v < list[KMAX - 1]) topk_insert<KMAX>(list, v);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (consumers_sync_or(failed)) break;
            if (c.last) {
                block_merge_write<KMAX>(list, k, out_ids + q * k, out_d + q * k, red);
                done_q = c.qi + gridDim.x;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (failed || abort_sh) {
            // a wait ran out: empty results for this CTA's queries not written yet
            for (int64_t r = done_q; r < nq; r += gridDim.x)
                for (int t = tid; t < k; t += PLAIN_CONSUMERS) {
                    out_ids[query_of(r) * k + t] = -1;
                    out_d[query_of(r) * k + t] = __uint_as_float(0x7F800000u);
                }
        }
    }
    __syncthreads();
}

template <int F, int KMAX, bool EXCL>
static int launch_plain_t(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad, const float* Y,
                          int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC, int k,
                          const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist,
                          int64_t grid, int num_sms, int64_t* out_ids, float* out_d, uint32_t* status,
                          cudaStream_t st)
{
    const int smem = PLAIN_STAGES * PLAIN_STAGE_FLOATS * 4;
    auto kern = plain_scan_kernel<F, KMAX, EXCL>;
    static int per_sm = 0;  // resident CTAs per SM of this instantiation
    if (!per_sm) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, PLAIN_THREADS, smem) != cudaSuccess || n < 1) n = 1;
        cudaGetLastError();
        per_sm = n;
    }
    // persistent: one wave of resident CTAs walks the queries
    const int64_t cap = int64_t(num_sms) * per_sm;
    const int64_t g = grid < cap ? grid : cap;
    kern<<<unsigned(g), PLAIN_THREADS, smem, st>>>(xs, offsets, perm, d_pad, Y, d, probes, P_eff, NC, k, query_src,
                                                   grid_w, radius, qlist, Q, out_ids, out_d, status,
                                                   g_plain_wait_budget);
    return count_launch();
}

template <int F, bool EXCL>
static int launch_plain_k(int k, const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad,
                          const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC,
                          const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist, int64_t grid,
                          int num_sms, int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st)
{
#define OSANN_PLAIN(KM)                                                                                      \
    return launch_plain_t<F, KM, EXCL>(xs, offsets, perm, d_pad, Y, d, Q, probes, P_eff, NC, k, query_src, grid_w, \
                                       radius, qlist, grid, num_sms, out_ids, out_d, status, st)
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
    // at most one CTA per query (a listed subset of unknown size: up to Q)
    const int64_t grid = Q;
#define OSANN_PLAIN_F(F, EX)                                                                                     \
    return launch_plain_k<F, EX>(k, xs, offsets, perm, d_pad, Y, d, Q, probes, P_eff, NC, query_src, grid_w, radius, \
                                 qlist, grid, num_sms, out_ids, out_d, status, st)
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
