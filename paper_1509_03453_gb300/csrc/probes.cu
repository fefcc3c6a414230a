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

// C(n, k) for k <= KM: the product formula when KM <= 4 (no table load; the
// products stay below 2^32 for n <= MAX_D = 256: 256 * 255 * 254 * 253 <
// 2^32), the table otherwise.
template <int KM>
__device__ __forceinline__ uint64_t Cs(const uint64_t* __restrict__ binom, int n, int k)
{
    if (KM <= 0 || KM > 4) return C(binom, n, k);
    if (n < 0 || k < 0 || k > n) return 0;
    const uint32_t m = uint32_t(n);
    switch (k) {
    case 0: return 1;
    case 1: return m;
    case 2: return m * (m - 1) / 2u;
    case 3: return m * (m - 1) * (m - 2) / 6u;
    default: return m * (m - 1) * (m - 2) * (m - 3) / 24u;
    }
}

// Smallest r' >= r with t < C(n - r' - 1, m - 1): the next member of the
// t-th m-subset (lexicographic) of {0..n-1} after value r - 1; t is reduced
// by the subsets skipped.  Bounded by n - m.
template <int KM>
__device__ __forceinline__ int next_member(const uint64_t* __restrict__ binom, uint64_t& t, int r, int n, int m)
{
    if (m == 1) {
        // every candidate value accounts for exactly one subset: step t values at once
        const uint64_t room = r < n - 1 ? uint64_t(n - 1 - r) : 0;
        const uint64_t step = t < room ? t : room;
        t -= step;
        return r + int(step);
    }
    while (r < n - m) {
        const uint64_t cnt = Cs<KM>(binom, n - r - 1, m - 1);
        if (t < cnt) break;
        t -= cnt;
        ++r;
    }
    return r;
}

// n (n-1) ... (n-k+1), the ordered selections of k of n (0 for k > n).
__device__ __forceinline__ uint64_t falling(int n, int k)
{
    if (k > n) return 0;
    uint64_t f = 1;
    for (int i = 0; i < k; ++i) f *= uint64_t(n - i);
    return f;
}

// ORDERED key (the members as a tuple in decreasing magnitude): the
// profile tree is the tree of ordered prefixes, so a tuple is at distance
// delta = L - (length of its common prefix with the query's tuple
// (i_1..i_L)).  Class delta keeps (i_1..i_(L-delta)); its next member has
// rank (0-based position in the query's order) in keep+1 .. d-1 (any but
// i_(keep+1)), each later one any unused rank in keep .. d-1; there are
// (n0-1) (n0-1)!/(n0-delta)! such tuples, n0 = d - keep.  Inside a class the
// rank tuple is lexicographic: position idx is unranked as a mixed-radix
// number whose m-th digit picks the digit-th unused rank.  Writes the
// members' ranks rk[0..L-1]; idx < nprof = d!/(d-L)! on entry.
template <int LM>
__device__ __forceinline__ void unrank_ordered(uint64_t idx, int d, int L, int (&rk)[LM])
{
    int delta = 0;
    for (; delta < L; ++delta) {
        const int n0 = d - L + delta;
        const uint64_t cnt = delta == 0 ? 1 : uint64_t(n0 - 1) * falling(n0 - 1, delta - 1);
        if (idx < cnt) break;
        idx -= cnt;
    }
    const int keep = L - delta;
    const int n0 = d - keep;
#pragma unroll
    for (int j = 0; j < LM; ++j)
        if (j < keep) rk[j] = j;
    for (int m = 0; m < delta; ++m) {
        // completions of the later positions, each choosing among the unused ranks
        const uint64_t f = falling(n0 - 1 - m, delta - 1 - m);
        const uint64_t digit = idx / f;
        idx -= digit * f;
        // the digit-th rank in keep (keep + 1 for the first member) .. d-1 not used yet
        int v = (m == 0 ? keep + 1 : keep) + int(digit);
        for (;;) {
            int below = 0;  // earlier members at ranks <= v, past the start of the range
#pragma unroll
            for (int t = 0; t < LM; ++t)
                if (t >= keep && t < keep + m && rk[t] <= v) ++below;
            const int target = (m == 0 ? keep + 1 : keep) + int(digit) + below;
            if (target == v) break;
            v = target;
        }
        rk[keep + m] = v;
    }
}

// Words per entry of the position table: the members' magnitude ranks as
// bytes (MAX_L of them), then the flip mask.
constexpr int PROBE_TAB_WORDS = MAX_L / 4 + 1;
constexpr int PROBE_SPAN = 4096;  // list positions per block of the probe kernel

// Which magnitude ranks the profile at list position p takes, and which of
// its members are sign-flipped, depend only on (d, L, p), not on the query:
// unrank every position once per search.  Table entry p: PROBE_TAB_WORDS
// words (ranks, flip mask).
template <int LC, bool ORD>
__global__ void __launch_bounds__(256) probe_ranks_kernel(int64_t P_eff, int d, int L,
                                                          const uint64_t* __restrict__ binom,
                                                          uint32_t* __restrict__ tab)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    if (LC > 0) L = LC;
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P_eff) return;
    uint64_t idx = uint64_t(p);
    const uint64_t nprof = ORD ? falling(d, L) : Cs<LC>(binom, d, L);
    uint32_t flip = 0;  // bit m: flip the member at position m of the ascending-|y| member list
    if (idx >= nprof) {
        idx -= nprof;
        for (int h = 1; h <= L; ++h) {
            const uint64_t per = Cs<LC>(binom, L, h);
            const uint64_t blk = nprof * per;
            if (idx < blk) {
                uint64_t fs = idx % per;
                idx /= per;
                int r = 0;
                for (int j = 0; j < h; ++j) {
                    r = next_member<LC>(binom, fs, r, L, h - j);
                    flip |= 1u << r;
                    ++r;
                }
                break;
            }
            idx -= blk;
        }
    }
    int rk[LM];  // member ranks (0-based positions into a query's order)
    if (ORD) {
        unrank_ordered<LM>(idx, d, L, rk);
    } else {
        // profile class delta, then the idx-th delta-subset of the ranks after keep
        int delta = 0;
        for (; delta < L; ++delta) {
            const uint64_t cnt = delta == 0 ? 1 : Cs<LC>(binom, d - L + delta - 1, delta);
            if (idx < cnt) break;
            idx -= cnt;
        }
        const int keep = L - delta;
        const int n = d - keep - 1;  // candidate ranks keep+1 .. d-1
        int r = 0;
#pragma unroll
        for (int j = 0; j < LM; ++j) {
            if (LC > 0 || j < L) {
                if (j < keep) {
                    rk[j] = j;
                } else {
                    r = next_member<LC>(binom, idx, r, n, L - j);
                    rk[j] = keep + 1 + r;
                    ++r;
                }
            }
        }
    }
    uint32_t w[PROBE_TAB_WORDS];
#pragma unroll
    for (int i = 0; i < PROBE_TAB_WORDS; ++i) w[i] = 0;
#pragma unroll
    for (int j = 0; j < LM; ++j)
        if (LC > 0 || j < L) w[j >> 2] |= uint32_t(rk[j]) << (8 * (j & 3));
    w[PROBE_TAB_WORDS - 1] = flip;
#pragma unroll
    for (int i = 0; i < PROBE_TAB_WORDS; ++i) tab[p * PROBE_TAB_WORDS + i] = w[i];
}

// LC: L as a compile-time constant (1..4), or 0 for a runtime L <= MAX_L.
// WIDE: 128-bit cone ids looked up in the second-level table (pm).
// Q counts the rows of qorder/qsign: pm.M per query with clusters.  Block
// (x, y) serves row x, positions y * PROBE_SPAN + threadIdx.x + 256 i (one
// thread per (row, position), up to PROBE_SPAN / 256 positions per thread): the
// position's ranks and flips from the table, mapped through the row's
// magnitude order and signs, staged in shared memory once per block.
template <int LC, bool WIDE>
__global__ void __launch_bounds__(256) probes_kernel(const uint8_t* __restrict__ qorder,
                                                     const uint32_t* __restrict__ qsign, int64_t Q, int d, int L,
                                                     int64_t P_eff, const uint64_t* __restrict__ binom,
                                                     const uint32_t* __restrict__ tab,
                                                     uint32_t* __restrict__ probes, uint64_t* __restrict__ partial,
                                                     int k, const ProbeMap pm)
{
    constexpr int LM = LC > 0 ? LC : MAX_L;
    if (LC > 0) L = LC;
    __shared__ uint8_t ord[MAX_D];
    __shared__ uint32_t sg[MAX_D / 32];
    const int64_t q = blockIdx.x;  // row of qorder/qsign
    for (int i = threadIdx.x; i < d; i += blockDim.x) ord[i] = qorder[q * int64_t(d) + i];
    if (threadIdx.x < MAX_D / 32) sg[threadIdx.x] = qsign[q * (MAX_D / 32) + threadIdx.x];
    __syncthreads();
    const int64_t pend = int64_t(blockIdx.y + 1) * PROBE_SPAN < P_eff ? int64_t(blockIdx.y + 1) * PROBE_SPAN : P_eff;
#pragma unroll 4
    for (int64_t posn = int64_t(blockIdx.y) * PROBE_SPAN + threadIdx.x; posn < pend; posn += blockDim.x) {
        const int64_t t = q * P_eff + posn;
        uint32_t w[PROBE_TAB_WORDS];
#pragma unroll
        for (int i = 0; i < PROBE_TAB_WORDS; ++i)
            if (i < (LM + 3) / 4 || i == PROBE_TAB_WORDS - 1) w[i] = __ldg(tab + posn * PROBE_TAB_WORDS + i);
        const uint32_t flip = w[PROBE_TAB_WORDS - 1];
        int rk[LM];  // member ranks (0-based positions into the query's order)
        int cm[LM];  // member components
#pragma unroll
        for (int j = 0; j < LM; ++j)
            if (LC > 0 || j < L) {
                rk[j] = int((w[j >> 2] >> (8 * (j & 3))) & 0xFFu);
                cm[j] = ord[rk[j]];
            }
        // cone id of the profile with the query's signs (and the chosen flips)
        uint64_t rank = 0;
        u128 rank_w = 0;
        uint32_t code = 0;
#pragma unroll
        for (int j = 0; j < LM; ++j) {
            if (LC > 0 || j < L) {
                int pos = 0, asc = 0;
#pragma unroll
                for (int u = 0; u < LM; ++u) {
                    if (LC > 0 || u < L) {
                        pos += cm[u] < cm[j] ? 1 : 0;  // ascending component index
                        asc += rk[u] > rk[j] ? 1 : 0;  // ascending magnitude
                    }
                }
                uint32_t bit = (sg[cm[j] >> 5] >> (cm[j] & 31)) & 1u;
                bit ^= (flip >> asc) & 1u;
                if (pm.ordered) {
                    // tuple position j: c_j = cm[j] minus the earlier members below it
                    int below = 0;
                    uint64_t after = 1;
#pragma unroll
                    for (int u = 0; u < LM; ++u) {
                        if (u < j && cm[u] < cm[j]) ++below;
                        if (u > j && (LC > 0 || u < L)) after *= uint64_t(d - u);
                    }
                    rank += uint64_t(cm[j] - below) * after;
                    code |= bit << (L - 1 - j);
                } else {
                    if (WIDE) rank_w += binom_wide(pm.binom_w, cm[j], pos + 1);
                    else rank += Cs<LC>(binom, cm[j], pos + 1);
                    code |= bit << (L - 1 - pos);
                }
            }
        }
        const uint32_t cl = pm.vcl ? pm.vcl[q] : 0u;
        uint32_t cone;
        if (WIDE) {
            u128 id = (rank_w << L) | u128(code);
            if (pm.vcl) id += u128(cl) * ((u128(pm.ncc_hi) << 64) | u128(pm.ncc_lo));
            cone = cone_lookup(wide_words(id), pm.ukeys, pm.htab, pm.hmask, pm.sentinel);
        } else {
            cone = uint32_t((rank << L) | code) + cl * uint32_t(pm.ncc_lo);
        }
        // slot of this position in its query's list: query q / M, position
        // (q % M) * P_eff + p; its flat index is t either way
        probes[t] = cone;
        if (partial)
            for (int j = 0; j < k; ++j) partial[t * k + j] = EMPTY_DI;
    }
}

size_t probe_table_bytes(int64_t P_eff) { return size_t(P_eff > 0 ? P_eff : 1) * PROBE_TAB_WORDS * 4; }

int launch_probes(const uint8_t* qorder, const uint32_t* qsign, int64_t Q, int d, int L, int64_t P_eff,
                  const uint64_t* binom, uint32_t* tab, uint32_t* probes, uint64_t* partial, int k, cudaStream_t st,
                  const ProbeMap& pm)
{
    const int64_t n = Q * P_eff;
    if (n == 0) return 0;
    {
        const unsigned gt = unsigned((P_eff + 255) / 256);
#define OSANN_RANKS(LC, O) probe_ranks_kernel<LC, O><<<gt, 256, 0, st>>>(P_eff, d, L, binom, tab)
        if (pm.ordered) {
            switch (L) {
            case 1: OSANN_RANKS(1, true); break;
            case 2: OSANN_RANKS(2, true); break;
            case 3: OSANN_RANKS(3, true); break;
            default: OSANN_RANKS(0, true); break;
            }
        } else {
            switch (L) {
            case 1: OSANN_RANKS(1, false); break;
            case 2: OSANN_RANKS(2, false); break;
            case 3: OSANN_RANKS(3, false); break;
            case 4: OSANN_RANKS(4, false); break;
            default: OSANN_RANKS(0, false); break;
            }
        }
#undef OSANN_RANKS
        const int rc = count_launch();
        if (rc) return rc;
    }
    if (P_eff > int64_t(65535) * PROBE_SPAN || Q > int64_t(0x7FFFFFFF)) return -2;  // grid limits
    const dim3 g(unsigned(Q), unsigned((P_eff + PROBE_SPAN - 1) / PROBE_SPAN));
#define OSANN_PROBES(LC, W) \
    probes_kernel<LC, W><<<g, 256, 0, st>>>(qorder, qsign, Q, d, L, P_eff, binom, tab, probes, partial, k, pm)
    if (pm.htab) {
        OSANN_PROBES(0, true);
        return count_launch();
    }
    switch (L) {
    case 1: OSANN_PROBES(1, false); break;
    case 2: OSANN_PROBES(2, false); break;
    case 3: OSANN_PROBES(3, false); break;
    case 4: OSANN_PROBES(4, false); break;
    default: OSANN_PROBES(0, false); break;
    }
#undef OSANN_PROBES
    return count_launch();
}

}  // namespace osann
