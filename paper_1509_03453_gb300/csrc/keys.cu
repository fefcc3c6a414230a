// Cone keys of data vectors and magnitude orders of query vectors.
//
// Sec. 2 of the paper: a vector's profile is the unordered set of its G
// largest-magnitude components, its cone the profile plus the signs of those
// components.  Here G is called L and the key is
//     key = rank(S) * 2^L + signcode,
//     rank(S)  = sum_j C(s_j, j+1) over the members sorted ascending (s_0 < s_1 ...),
//     signcode = sum_j [x_{s_j} >= 0] * 2^(L-1-j),
// ties between equal magnitudes going to the lower component index.
// Queries additionally need the full order i_1..i_K of Sec. 3-B (indices by
// decreasing magnitude), from which the probe kernel derives the
// neighbouring cones, and their sign bits.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

// Selection key of one component: |x| bits in the high word, then the
// complement of the component index (so that equal magnitudes prefer the
// lower index under max), then the sign bit.
__device__ __forceinline__ uint64_t sel_key(float x, int comp)
{
    uint32_t a = __float_as_uint(x) & 0x7FFFFFFFu;
    uint32_t lo = (uint32_t(MAX_D - 1 - comp) << 1) | (x >= 0.0f ? 1u : 0u);
    return (uint64_t(a) << 32) | lo;
}
__device__ __forceinline__ int sel_comp(uint64_t k) { return MAX_D - 1 - int((uint32_t(k) >> 1) & 0x3FFu); }
__device__ __forceinline__ uint32_t sel_sign(uint64_t k) { return uint32_t(k) & 1u; }

__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7F800000u) != 0x7F800000u; }

// Cone id from the L selected (component, sign) pairs, in any order.  LC is
// L when it is a compile-time constant (the loops then unroll to exactly L),
// or 0 for a runtime L up to MAX_L.
template <int LC>
__device__ __forceinline__ uint32_t cone_from_members(const int (&comp)[MAX_L], const uint32_t (&sgn)[MAX_L], int L,
                                                      const uint64_t* __restrict__ binom)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    uint64_t rank = 0;
    uint32_t code = 0;
#pragma unroll
    for (int j = 0; j < LM; ++j) {
        if (LC > 0 || j < L) {
            int pos = 0;  // position of member j in ascending component order
#pragma unroll
            for (int t = 0; t < LM; ++t)
                if ((LC > 0 || t < L) && comp[t] < comp[j]) ++pos;
            rank += __ldg(binom + comp[j] * (MAX_L + 1) + pos + 1);
            code |= sgn[j] << (L - 1 - pos);
        }
    }
    return uint32_t((rank << L) | code);
}

// The same id in 128 bits (N_C >= 2^31: the second-level table).
template <int LC>
__device__ __forceinline__ uint4 cone_wide_from_members(const int (&comp)[MAX_L], const uint32_t (&sgn)[MAX_L], int L,
                                                        const ulonglong2* __restrict__ binom_w)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    u128 rank = 0;
    uint32_t code = 0;
#pragma unroll
    for (int j = 0; j < LM; ++j) {
        if (LC > 0 || j < L) {
            int pos = 0;
#pragma unroll
            for (int t = 0; t < LM; ++t)
                if ((LC > 0 || t < L) && comp[t] < comp[j]) ++pos;
            rank += binom_wide(binom_w, comp[j], pos + 1);
            code |= sgn[j] << (L - 1 - pos);
        }
    }
    return wide_words((rank << L) | u128(code));
}

// ORDERED key: the members as a tuple in decreasing magnitude (comp[0] the
// largest), numbered lexicographically among the L-permutations of the d
// components, rank = sum_j c_j (d-1-j)!/(d-L)! with c_j = comp[j] minus the
// number of earlier members below it; the sign of member j at bit L-1-j.
// N_C = d!/(d-L)! 2^L < 2^31 (checked on the host), so rank fits 64 bits.
template <int LC>
__device__ __forceinline__ uint32_t ordered_from_members(const int (&comp)[MAX_L], const uint32_t (&sgn)[MAX_L],
                                                         int L, int d)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    uint64_t rank = 0;
    uint32_t code = 0;
#pragma unroll
    for (int j = 0; j < LM; ++j) {
        if (LC > 0 || j < L) {
            int below = 0;
#pragma unroll
            for (int t = 0; t < LM; ++t)
                if (t < j && comp[t] < comp[j]) ++below;
            uint64_t after = 1;  // (d-1-j)!/(d-L)!: ways to fill the later positions
#pragma unroll
            for (int m = 0; m < LM; ++m)
                if (m > j && (LC > 0 || m < L)) after *= uint64_t(d - m);
            rank += uint64_t(comp[j] - below) * after;
            code |= sgn[j] << (L - 1 - j);
        }
    }
    return uint32_t((rank << L) | code);
}

// Store the key of one row: a direct-table id, or (WIDE) a 128-bit id; ORD:
// the ORDERED key (direct table only).  comp[] lists the members by
// decreasing magnitude (ties: the lower component first).
template <int LC, bool WIDE, bool ORD>
__device__ __forceinline__ void store_key(int64_t row, const int (&comp)[MAX_L], const uint32_t (&sgn)[MAX_L], int L,
                                          int d, const uint64_t* __restrict__ binom,
                                          const ulonglong2* __restrict__ binom_w, uint32_t* __restrict__ keys,
                                          uint4* __restrict__ wkeys)
{
    if (ORD) keys[row] = ordered_from_members<LC>(comp, sgn, L, d);
    else if (WIDE) wkeys[row] = cone_wide_from_members<LC>(comp, sgn, L, binom_w);
    else keys[row] = cone_from_members<LC>(comp, sgn, L, binom);
}

// Vector path (d % 4 == 0, 16-byte aligned rows): one lane per row.  The
// lane streams its row in pieces of up to KC float4 (the first line fetch
// brings the piece's cache lines into L1 for the rest of the warp's loads)
// and keeps the L largest magnitudes in a sorted register list: one 32-bit
// compare per component, an insertion only when the component can enter.
template <int LC, bool WIDE, bool ORD>
__global__ void __launch_bounds__(256) data_keys_row_kernel(const float* __restrict__ X, int64_t N, int d, int L,
                                                           const uint64_t* __restrict__ binom,
                                                           const ulonglong2* __restrict__ binom_w,
                                                           uint32_t* __restrict__ keys, uint4* __restrict__ wkeys,
                                                           uint32_t* __restrict__ status,
                                                           uint32_t* __restrict__ maxn2_bits)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    constexpr int KC = 8;  // float4 per piece
    const int lane = threadIdx.x & 31;
    const int n4 = d >> 2;
    bool bad = false;
    float nmax = 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < N; row += stride) {
        const float4* xr = reinterpret_cast<const float4*>(X + row * int64_t(d));
        // the L largest magnitudes so far, descending, with their components and
        // sign bits (1: x >= 0); -1 = empty.  Components arrive in increasing
        // index order, so an incoming one never displaces an earlier one of equal
        // magnitude (the lower component first): a strict 32-bit magnitude
        // compare places it, and the entries after it shift down.
        int mag[LM], cix[LM];
        uint32_t csg[LM];
#pragma unroll
        for (int r = 0; r < LM; ++r) {
            mag[r] = -1;
            cix[r] = 0;
            csg[r] = 0;
        }
        int lastmag = -1;  // the L-th entry's magnitude: only a larger one enters
        uint32_t amax = 0;  // largest magnitude bits of the row: >= 0x7F800000 iff non-finite
        float nsq = 0.0f;
        for (int c0 = 0; c0 < n4; c0 += KC) {
            float4 t[KC];
#pragma unroll
            for (int f = 0; f < KC; ++f) t[f] = c0 + f < n4 ? __ldg(xr + c0 + f) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int f = 0; f < KC; ++f) {
                if (c0 + f < n4) {
                    const float x4[4] = {t[f].x, t[f].y, t[f].z, t[f].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float x = x4[e];
                        const uint32_t au = __float_as_uint(x) & 0x7FFFFFFFu;
                        amax = au > amax ? au : amax;
                        nsq = fmaf(x, x, nsq);
                        if (int(au) > lastmag) {
                            // insertion: the first entry with a smaller magnitude and
                            // every one after it move down one place
                            int m = int(au), ci = 4 * (c0 + f) + e;
                            uint32_t sg = x >= 0.0f ? 1u : 0u;
                            bool placed = false;
#pragma unroll
                            for (int r = 0; r < LM; ++r) {
                                if ((LC > 0 || r < L) && (placed || m > mag[r])) {
                                    placed = true;
                                    const int tm = mag[r], tc = cix[r];
                                    const uint32_t ts = csg[r];
                                    mag[r] = m;
                                    cix[r] = ci;
                                    csg[r] = sg;
                                    m = tm;
                                    ci = tc;
                                    sg = ts;
                                }
                            }
                            lastmag = mag[LM - 1];
                            if (LC == 0) {
#pragma unroll
                                for (int r = 0; r < LM; ++r)
                                    if (r == L - 1) lastmag = mag[r];
                            }
                        }
                    }
                }
            }
        }
        bad |= amax >= 0x7F800000u;
        int comp[MAX_L];
        uint32_t sgn[MAX_L];
#pragma unroll
        for (int r = 0; r < MAX_L; ++r) {
            comp[r] = 0;
            sgn[r] = 0;
        }
#pragma unroll
        for (int r = 0; r < LM; ++r)
            if (LC > 0 || r < L) {
                comp[r] = cix[r];
                sgn[r] = csg[r];
            }
        store_key<LC, WIDE, ORD>(row, comp, sgn, L, d, binom, binom_w, keys, wkeys);
        nmax = fmaxf(nmax, nsq);  // non-finite rows are reported separately
    }
    if (maxn2_bits) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        // nonnegative floats order like their bits
        if (lane == 0 && nmax > 0.0f && finite_f(nmax)) atomicMax(maxn2_bits, __float_as_uint(nmax));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE_DATA);
}

// One group of LPV lanes per row.  VEC: d % 4 == 0 and 16-byte aligned rows,
// lane l holds float4 number l, l+LPV (128-bit loads); else lane l holds the
// scalars l, l+32, ... (LPV = 32).  At most 8 values per lane (d <= 256).
template <int LPV, bool VEC, int LC, bool WIDE, bool ORD>
__global__ void __launch_bounds__(256) data_keys_kernel(const float* __restrict__ X, int64_t N, int d, int L,
                                                       const uint64_t* __restrict__ binom,
                                                       const ulonglong2* __restrict__ binom_w,
                                                       uint32_t* __restrict__ keys, uint4* __restrict__ wkeys,
                                                       uint32_t* __restrict__ status,
                                                       uint32_t* __restrict__ maxn2_bits)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    const int lane = threadIdx.x & 31;
    const int glane = lane & (LPV - 1);
    const int64_t gid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / LPV;
    const int64_t ngroups = int64_t(gridDim.x) * blockDim.x / LPV;
    bool bad = false;
    float nmax = 0.0f;  // largest squared row norm seen by this lane's group
    // rows are taken two at a time per group (both loads in flight before
    // either is processed); every group of the warp runs the same trip count
    // so shuffles stay converged
    const int64_t iters = (N + 2 * ngroups - 1) / (2 * ngroups);
    for (int64_t it = 0; it < iters; ++it) {
        uint64_t v[2][8];
        int64_t rows[2];
        float nsq[2] = {0.0f, 0.0f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t row = gid + (2 * it + h) * ngroups;
            rows[h] = row;
            const bool live = row < N;
#pragma unroll
            for (int f = 0; f < 8; ++f) v[h][f] = 0;  // 0 = empty slot (real keys are > 0)
            if (VEC) {
                const float4* xr = reinterpret_cast<const float4*>(X + (live ? row : 0) * int64_t(d));
                const int n4 = d >> 2;
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    int i4 = glane + f * LPV;
                    if (live && i4 < n4) {
                        float4 t = __ldg(xr + i4);
                        bad |= !(finite_f(t.x) && finite_f(t.y) && finite_f(t.z) && finite_f(t.w));
                        nsq[h] = fmaf(t.x, t.x, fmaf(t.y, t.y, fmaf(t.z, t.z, fmaf(t.w, t.w, nsq[h]))));
                        v[h][4 * f + 0] = sel_key(t.x, 4 * i4 + 0);
                        v[h][4 * f + 1] = sel_key(t.y, 4 * i4 + 1);
                        v[h][4 * f + 2] = sel_key(t.z, 4 * i4 + 2);
                        v[h][4 * f + 3] = sel_key(t.w, 4 * i4 + 3);
                    }
                }
            } else {
                const float* xr = X + (live ? row : 0) * int64_t(d);
#pragma unroll
                for (int f = 0; f < 8; ++f) {
                    int c = glane + f * 32;
                    if (live && c < d) {
                        float t = __ldg(xr + c);
                        bad |= !finite_f(t);
                        nsq[h] = fmaf(t, t, nsq[h]);
                        v[h][f] = sel_key(t, c);
                    }
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int comp[MAX_L];
            uint32_t sgn[MAX_L];
#pragma unroll
            for (int r = 0; r < MAX_L; ++r) {
                comp[r] = 0;
                sgn[r] = 0;
            }
#pragma unroll
            for (int r = 0; r < LM; ++r) {
                if (LC > 0 || r < L) {
                    uint64_t best = 0;
#pragma unroll
                    for (int f = 0; f < 8; ++f) best = v[h][f] > best ? v[h][f] : best;
#pragma unroll
                    for (int m = LPV / 2; m > 0; m >>= 1) {
                        uint64_t o = shfl_xor_u64(best, m);
                        best = o > best ? o : best;
                    }
#pragma unroll
                    for (int f = 0; f < 8; ++f)
                        if (v[h][f] == best) v[h][f] = 0;  // taken (keys are unique per row)
                    comp[r] = sel_comp(best);
                    sgn[r] = sel_sign(best);
                }
            }
            if (rows[h] < N && glane == 0)
                store_key<LC, WIDE, ORD>(rows[h], comp, sgn, L, d, binom, binom_w, keys, wkeys);
#pragma unroll
            for (int m = LPV / 2; m > 0; m >>= 1) nsq[h] += __shfl_xor_sync(0xffffffffu, nsq[h], m);
            nmax = fmaxf(nmax, nsq[h]);  // non-finite rows are reported separately
        }
    }
    if (maxn2_bits) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        // nonnegative floats order like their bits
        if (lane == 0 && nmax > 0.0f && finite_f(nmax)) atomicMax(maxn2_bits, __float_as_uint(nmax));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE_DATA);
}

// One warp per query: full magnitude order (rank -> component, u8) and sign
// bits (bit c of word c/32 set when y_c >= 0).
__global__ void __launch_bounds__(128) query_order_kernel(const float* __restrict__ Y, int64_t Q, int d,
                                                          uint8_t* __restrict__ qorder,
                                                          uint32_t* __restrict__ qsign,
                                                          uint32_t* __restrict__ status)
{
    __shared__ uint64_t sk[4][MAX_D];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = int64_t(blockIdx.x) * 4 + warp;
    if (q >= Q) return;  // whole warp leaves together
    const float* y = Y + q * int64_t(d);
    bool bad = false;
    for (int c = lane; c < d; c += 32) {
        float t = y[c];
        bad |= !finite_f(t);
        sk[warp][c] = sel_key(t, c) | 1u;  // sign bit neutralised: order uses |y| and index only
    }
    for (int w = 0; w < (d + 31) / 32; ++w) {
        int c = w * 32 + lane;
        bool pos = c < d ? (y[c] >= 0.0f) : false;
        unsigned b = __ballot_sync(0xffffffffu, pos);
        if (lane == 0) qsign[q * (MAX_D / 32) + w] = b;
    }
    __syncwarp();
    for (int c = lane; c < d; c += 32) {
        uint64_t me = sk[warp][c];
        int rank = 0;
        for (int j = 0; j < d; ++j) rank += sk[warp][j] > me ? 1 : 0;
        qorder[q * int64_t(d) + rank] = uint8_t(c);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE_QUERY);
}

// Coordinates on a rotated basis (Sec. 3-D) or a projection on m <= d
// components (Sec. 4-B): out[i][r] = (sum_j P[r][j] x_i[j]) - off[r],
// the sum in fp32 fused multiply-adds in order j = 0, 1, ... from 0, then one
// subtraction (off may be null) -- the order the keys' parity depends on.
// A CTA takes ROT_ROWS rows; P is held transposed in shared memory (lanes
// read consecutive outputs of one column: no bank conflicts), the rows'
// inputs are broadcast.  d <= 128.
constexpr int ROT_ROWS = 32;

__global__ void __launch_bounds__(256) rotate_rows_kernel(const float* __restrict__ Pm, const float* __restrict__ off,
                                                          const float* __restrict__ X, int64_t n, int d, int m,
                                                          float* __restrict__ out)
{
    extern __shared__ float rsh[];
    float* Pt = rsh;              // d x m, Pt[j * m + r] = P[r][j]
    float* xt = rsh + d * m;      // ROT_ROWS x d
    for (int e = threadIdx.x; e < m * d; e += blockDim.x) {
        const int r = e / d, j = e - r * d;
        Pt[j * m + r] = Pm[e];
    }
    for (int64_t base = int64_t(blockIdx.x) * ROT_ROWS; base < n; base += int64_t(gridDim.x) * ROT_ROWS) {
        const int rows = n - base < ROT_ROWS ? int(n - base) : ROT_ROWS;
        __syncthreads();
        for (int e = threadIdx.x; e < rows * d; e += blockDim.x) xt[e] = X[base * d + e];
        __syncthreads();
        for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
            const int i = e / m, r = e - i * m;
            const float* x = xt + i * d;
            float acc = 0.0f;
            for (int j = 0; j < d; ++j) acc = fmaf(Pt[j * m + r], x[j], acc);
            out[base * m + e] = off ? acc - off[r] : acc;
        }
    }
}

int launch_rotate_rows(const float* Pm, const float* off, const float* X, int64_t n, int d, int m, float* out,
                       cudaStream_t st, int num_sms)
{
    if (n == 0) return 0;
    if (d > 128 || m < 1 || m > d) return -2;  // the transposed basis must fit shared memory
    const size_t smem = size_t(d) * m * 4 + size_t(ROT_ROWS) * d * 4;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rotate_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(128 * 128 * 4 + ROT_ROWS * 128 * 4));
        attr = true;
    }
    int64_t blocks = (n + ROT_ROWS - 1) / ROT_ROWS;
    if (blocks > int64_t(num_sms) * 8) blocks = int64_t(num_sms) * 8;
    rotate_rows_kernel<<<unsigned(blocks), 256, smem, st>>>(Pm, off, X, n, d, m, out);
    return count_launch();
}

// Largest squared row norm of X (fp32 sums, any order: it only sizes the fp16
// scale and a norm bound, both with slack), as float bits for atomicMax.
__global__ void __launch_bounds__(256) row_norm_max_kernel(const float* __restrict__ X, int64_t n, int d,
                                                           uint32_t* __restrict__ maxn2_bits)
{
    float best = 0.0f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < n; row += stride) {
        const float* x = X + row * d;
        float s = 0.0f;
        for (int j = 0; j < d; ++j) s = fmaf(x[j], x[j], s);
        best = fmaxf(best, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > 0.0f && finite_f(best)) atomicMax(maxn2_bits, __float_as_uint(best));
}

int launch_row_norm_max(const float* X, int64_t n, int d, uint32_t* maxn2_bits, cudaStream_t st, int num_sms)
{
    if (n == 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > int64_t(num_sms) * 8) blocks = int64_t(num_sms) * 8;
    row_norm_max_kernel<<<unsigned(blocks), 256, 0, st>>>(X, n, d, maxn2_bits);
    return count_launch();
}

template <int LC, bool WIDE = false, bool ORD = false>
static void launch_keys_lc(bool vec, dim3 g, dim3 b, cudaStream_t st, const float* X, int64_t N, int d, int L,
                           const uint64_t* binom, const ulonglong2* binom_w, uint32_t* keys, uint4* wkeys,
                           uint32_t* status, uint32_t* maxn2)
{
    if (vec)
        data_keys_row_kernel<LC, WIDE, ORD><<<g, b, 0, st>>>(X, N, d, L, binom, binom_w, keys, wkeys, status, maxn2);
    else
        data_keys_kernel<32, false, LC, WIDE, ORD><<<g, b, 0, st>>>(X, N, d, L, binom, binom_w, keys, wkeys, status,
                                                                     maxn2);
}

int launch_data_keys(const float* X, int64_t N, int d, int L, const uint64_t* binom, uint32_t* keys,
                     uint32_t* status, uint32_t* maxn2_bits, cudaStream_t st, int num_sms,
                     const ulonglong2* binom_w, uint4* wkeys, bool ordered)
{
    if (N == 0) return 0;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const int threads = 256;
    // vector path: one lane per row; scalar path: a warp per row
    int64_t blocks = vec ? (N + threads - 1) / threads : (N * 32 + threads - 1) / threads;
    const int64_t cap = int64_t(num_sms) * (vec ? 8 : 16);
    if (blocks > cap) blocks = cap;
    const dim3 g(static_cast<unsigned>(blocks)), b(static_cast<unsigned>(threads));
    if (wkeys) {
        // 128-bit ids: one instantiation with a runtime L
        launch_keys_lc<0, true>(vec, g, b, st, X, N, d, L, binom, binom_w, nullptr, wkeys, status, maxn2_bits);
        return count_launch();
    }
    if (ordered) {
        switch (L) {
        case 1: launch_keys_lc<1, false, true>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
        case 2: launch_keys_lc<2, false, true>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
        case 3: launch_keys_lc<3, false, true>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
        default: launch_keys_lc<0, false, true>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
        }
        return count_launch();
    }
    switch (L) {
    case 1: launch_keys_lc<1>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
    case 2: launch_keys_lc<2>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
    case 3: launch_keys_lc<3>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
    case 4: launch_keys_lc<4>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
    default: launch_keys_lc<0>(vec, g, b, st, X, N, d, L, binom, nullptr, keys, nullptr, status, maxn2_bits); break;
    }
    return count_launch();
}

int launch_query_order(const float* Y, int64_t Q, int d, uint8_t* qorder, uint32_t* qsign, uint32_t* status,
                       cudaStream_t st)
{
    if (Q == 0) return 0;
    query_order_kernel<<<unsigned((Q + 3) / 4), 128, 0, st>>>(Y, Q, d, qorder, qsign, status);
    return count_launch();
}

}  // namespace osann
