// ROSANNA+ (Sec. 4-B): the data are clustered off line by k-means (the
// centroids are an input); every point belongs to its nearest centroid and is
// hashed by its residual x - c; a query visits its M nearest clusters, in
// each the cones of its residual y - c.  The index stores the composite cone
// id  cluster * N_C + cone(residual),  so one CSR table (direct, or the
// second-level table when K N_C >= 2^31) holds all clusters and every scan
// path runs unchanged on a probe list that concatenates the query's M
// per-cluster lists, nearest cluster first.
//
// "Nearest" is decided by the canonical fp32 squared distance of
// osann_device.cuh (padded float4 pieces, adjacent-pairwise tree), ties to
// the lower centroid index, so that every path and the oracle take the same
// integer decisions.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

// Piece j (components 4j .. 4j+3, zero past d) of a row that need not be
// padded or 16-byte aligned.
__device__ __forceinline__ float4 load_piece(const float* __restrict__ row, int d, int j, bool vec)
{
    const int c = 4 * j;
    if (vec) return c < d ? __ldg(reinterpret_cast<const float4*>(row) + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    return make_float4(c + 0 < d ? __ldg(row + c + 0) : 0.f, c + 1 < d ? __ldg(row + c + 1) : 0.f,
                       c + 2 < d ? __ldg(row + c + 2) : 0.f, c + 3 < d ? __ldg(row + c + 3) : 0.f);
}

// One warp per vector.  Lanes form groups of NF (= d_pad / 4 pieces, one
// piece per lane); each group takes one centroid per step, so 32 / NF
// centroids are compared at once.  The group's leader keeps a register list
// of the M best (distance, index) pairs; the leaders' lists are merged at
// the end.  C is K x d_pad (zero padded).  out[v * M + j], nearest first.
template <int NF, int KMAX>
__global__ void __launch_bounds__(256) nearest_centroids_kernel(const float* __restrict__ X, int64_t n, int d,
                                                                const float* __restrict__ C, int K, int M,
                                                                uint32_t* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t v = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;  // whole warp
    const int gl = lane % NF, grp = lane / NF;
    constexpr int GROUPS = 32 / NF;
    const float* xr = X + v * int64_t(d);
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const float4 xp = load_piece(xr, d, gl, vec);
    const int d_pad = 4 * NF;
    uint64_t list[KMAX];
    topk_init<KMAX>(list, M);
    for (int c0 = 0; c0 < K; c0 += GROUPS) {
        const int c = c0 + grp;
        float dist = INFINITY;
        if (c < K) dist = sq4(xp, __ldg(reinterpret_cast<const float4*>(C + int64_t(c) * d_pad) + gl));
        dist = lane_tree(dist, NF);  // groups of NF adjacent lanes: the canonical tree
        if (c < K && gl == 0) {
            const uint64_t key = pack_di(dist, uint32_t(c));
            if (key < list[KMAX - 1]) topk_insert<KMAX>(list, key);
        }
    }
    for (int j = 0; j < M; ++j) {
        const uint64_t head = gl == 0 ? topk_head<KMAX>(list, M) : EMPTY_DI;
        const uint64_t best = warp_min_u64(head);
        if (gl == 0 && head == best) topk_remove<KMAX>(list, M, best);
        if (lane == 0) out[v * M + j] = di_id(best);
    }
}

// out[(v * M + j) * d + e] = X[v][e] - C[idx[v * M + j]][e]  (fp32).
__global__ void __launch_bounds__(256) residual_rows_kernel(const float* __restrict__ X, int64_t n, int d,
                                                            const float* __restrict__ C, int d_pad,
                                                            const uint32_t* __restrict__ idx, int M,
                                                            float* __restrict__ out)
{
    const int64_t total = n * M * int64_t(d);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t vr = t / d;  // residual row v * M + j
        const int e = int(t - vr * d);
        const int64_t vi = vr / M;
        out[t] = X[vi * d + e] - C[int64_t(idx[vr]) * d_pad + e];
    }
}

// Composite ids: cone id of the residual plus cluster * N_C.
__global__ void __launch_bounds__(256) composite_keys_kernel(const uint32_t* __restrict__ asg, int64_t N,
                                                             uint64_t ncc_lo, uint64_t ncc_hi,
                                                             uint32_t* __restrict__ keys, uint4* __restrict__ wkeys)
{
    const u128 ncc = (u128(ncc_hi) << 64) | u128(ncc_lo);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        if (wkeys) wkeys[i] = wide_words(u128(asg[i]) * ncc + wide_value(wkeys[i]));
        else keys[i] = uint32_t(uint64_t(asg[i]) * ncc_lo + keys[i]);
    }
}

int launch_nearest_centroids(const float* X, int64_t n, int d, int d_pad, const float* C, int K, int M,
                             uint32_t* out, cudaStream_t st)
{
    if (n == 0) return 0;
    if (M < 1 || M > 32 || M > K || d_pad > 128 || d_pad < 16) return -2;
    const unsigned blocks = unsigned((n + 7) / 8);  // 8 warps per block
#define OSANN_NEAR(NF, KM) nearest_centroids_kernel<NF, KM><<<blocks, 256, 0, st>>>(X, n, d, C, K, M, out)
#define OSANN_NEAR_K(NF)             \
    if (M <= 1) OSANN_NEAR(NF, 1);   \
    else if (M <= 4) OSANN_NEAR(NF, 4); \
    else if (M <= 16) OSANN_NEAR(NF, 16); \
    else OSANN_NEAR(NF, 32);
    switch (d_pad / 4) {
    case 4: OSANN_NEAR_K(4); break;
    case 8: OSANN_NEAR_K(8); break;
    case 16: OSANN_NEAR_K(16); break;
    default: OSANN_NEAR_K(32); break;
    }
#undef OSANN_NEAR_K
#undef OSANN_NEAR
    return count_launch();
}

int launch_residual_rows(const float* X, int64_t n, int d, const float* C, int d_pad, const uint32_t* idx, int M,
                         float* out, cudaStream_t st, int num_sms)
{
    const int64_t total = n * M * int64_t(d);
    if (total == 0) return 0;
    int64_t blocks = (total + 255) / 256;
    if (blocks > int64_t(num_sms) * 16) blocks = int64_t(num_sms) * 16;
    residual_rows_kernel<<<unsigned(blocks), 256, 0, st>>>(X, n, d, C, d_pad, idx, M, out);
    return count_launch();
}

int launch_composite_keys(const uint32_t* asg, int64_t N, uint64_t ncc_lo, uint64_t ncc_hi, uint32_t* keys,
                          uint4* wkeys, cudaStream_t st, int num_sms)
{
    if (N == 0) return 0;
    int64_t blocks = (N + 255) / 256;
    if (blocks > int64_t(num_sms) * 8) blocks = int64_t(num_sms) * 8;
    composite_keys_kernel<<<unsigned(blocks), 256, 0, st>>>(asg, N, ncc_lo, ncc_hi, keys, wkeys);
    return count_launch();
}

}  // namespace osann
