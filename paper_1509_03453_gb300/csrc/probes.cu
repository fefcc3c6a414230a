// Ordered list of cones to visit per query (Algorithm 1, "find ordered list
// of cones"; neighbouring-cone order of Sec. 3-B).
//
// Let i_1..i_K be the query's components by decreasing magnitude.  A level-G
// profile S is at distance delta = G - max{g : {i_1..i_g} subset of S} from
// the query's profile.  The profiles at distance delta keep {i_1..i_(G-delta)}
// and take their other delta members from the ranks G-delta+2 .. K (there
// are C(K-G+delta-1, delta) of them).  The list visits delta = 0, 1, ..., G;
// inside a class, the substituted rank tuple in lexicographic order.  Each
// profile contributes the cone with the query's own signs.  After all C(K,G)
// profiles come the sign-flipped cones: h = 1..G flips, in profile order,
// the flipped members chosen as h-subsets (lexicographic) of the members
// sorted by |y| ascending.  All N_C cones appear exactly once.
//
// One thread per (query, probe position): the position is unranked directly,
// so any prefix of the list is produced without enumerating the ones before.
#include "osann_device.cuh"
#include "osann_launch.h"

namespace osann {

__device__ __forceinline__ uint64_t C(const uint64_t* __restrict__ binom, int n, int k)
{
    if (n < 0 || k < 0 || k > n) return 0;
    return __ldg(binom + n * (MAX_L + 1) + k);
}

// t-th m-subset of {0..n-1} in lexicographic order, written as ascending
// values into out[0..m-1].
__device__ __forceinline__ void unrank_lex(const uint64_t* __restrict__ binom, uint64_t t, int n, int m,
                                           int (&out)[MAX_L], int out_base)
{
    int r = 0;
    for (int j = 0; j < m; ++j) {
        // bounded: r never passes n - (m - j) for an in-range t
        while (r < n - (m - j)) {
            const uint64_t cnt = C(binom, n - r - 1, m - j - 1);
            if (t < cnt) break;
            t -= cnt;
            ++r;
        }
        out[out_base + j] = r;
        ++r;
    }
}

__global__ void __launch_bounds__(256) probes_kernel(const uint8_t* __restrict__ qorder,
                                                     const uint32_t* __restrict__ qsign, int64_t Q, int d, int L,
                                                     int64_t P_eff, const uint64_t* __restrict__ binom,
                                                     uint32_t* __restrict__ probes, uint64_t* __restrict__ partial,
                                                     int k)
{
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= Q * P_eff) return;
    const int64_t q = t / P_eff;
    uint64_t idx = uint64_t(t - q * P_eff);
    const uint8_t* ord = qorder + q * int64_t(d);
    const uint32_t* sg = qsign + q * (MAX_D / 32);

    const uint64_t nprof = C(binom, d, L);
    uint32_t flip = 0;  // bit m: flip the member at position m of the ascending-|y| member list
    if (idx >= nprof) {
        idx -= nprof;
        for (int h = 1; h <= L; ++h) {
            const uint64_t per = C(binom, L, h);
            const uint64_t blk = nprof * per;
            if (idx < blk) {
                const uint64_t fs = idx % per;
                idx /= per;
                int f[MAX_L];
                unrank_lex(binom, fs, L, h, f, 0);
                for (int j = 0; j < h; ++j) flip |= 1u << f[j];
                break;
            }
            idx -= blk;
        }
    }
    // unrank the profile: class delta, then the substituted rank tuple
    int rk[MAX_L];  // member ranks, 0-based positions into the query's order
    for (int j = 0; j < MAX_L; ++j) rk[j] = j;
    for (int delta = 0; delta <= L; ++delta) {
        const uint64_t cnt = delta == 0 ? 1 : C(binom, d - L + delta - 1, delta);
        if (idx < cnt) {
            const int keep = L - delta;
            for (int j = 0; j < keep; ++j) rk[j] = j;
            if (delta > 0) {
                unrank_lex(binom, idx, d - keep - 1, delta, rk, keep);
                for (int j = 0; j < delta; ++j) rk[keep + j] += keep + 1;
            }
            break;
        }
        idx -= cnt;
    }
    // cone id of the profile with the query's signs (and the chosen flips)
    uint64_t rank = 0;
    uint32_t code = 0;
    for (int j = 0; j < L; ++j) {
        const int cj = ord[rk[j]];
        int pos = 0, asc = 0;
        for (int u = 0; u < L; ++u) {
            const int cu = ord[rk[u]];
            pos += cu < cj ? 1 : 0;          // ascending component index
            asc += rk[u] > rk[j] ? 1 : 0;    // ascending magnitude
        }
        uint32_t bit = (sg[cj >> 5] >> (cj & 31)) & 1u;
        bit ^= (flip >> asc) & 1u;
        rank += C(binom, cj, pos + 1);
        code |= bit << (L - 1 - pos);
    }
    probes[t] = uint32_t((rank << L) | code);
    if (partial)
        for (int j = 0; j < k; ++j) partial[t * k + j] = EMPTY_DI;
}

int launch_probes(const uint8_t* qorder, const uint32_t* qsign, int64_t Q, int d, int L, int64_t P_eff,
                  const uint64_t* binom, uint32_t* probes, uint64_t* partial, int k, cudaStream_t st)
{
    const int64_t n = Q * P_eff;
    if (n == 0) return 0;
    probes_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(qorder, qsign, Q, d, L, P_eff, binom, probes, partial,
                                                             k);
    return count_launch();
}

}  // namespace osann
