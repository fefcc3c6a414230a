/*
 * osann_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * order-statistics cone-hash ANN search of Verdoliva, Cozzolino and Poggi,
 * "A reliable order-statistics-based approximate nearest neighbor search
 * algorithm" (ROSANNA): one basis (R = 1), and R bases (Algorithm 1 with
 * the union of its bases' cones) for the multi-basis search of Sec. 3-D.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library under paper_1509_03453_gb300/csrc) shares no code,
 * header, table or helper with this file, and never calls it.
 *
 * Every function follows the paper's steps in the paper's order and notation
 * (K = vector length, called d here; G = components used, called L here;
 * C = cones visited, called P here).  Distances are accumulated in double
 * precision.  No blocking, fusion or reordering is done beyond what the
 * definitions state.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *   - ties between equal magnitudes go to the lower component index;
 *   - profiles (unordered G-subsets) are numbered in colexicographic order,
 *     rank(S) = sum_j C(s_j, j+1) with s_0 < s_1 < ...;
 *   - the sign code of a cone puts the lowest component index in the most
 *     significant bit and counts zero (and -0.0) as positive (Fig. 2);
 *   - cone id = rank(S) * 2^G + sign code;
 *   - within one profile distance class the probe order is the lexicographic
 *     order of the substituted rank tuple; each probed profile contributes the
 *     cone carrying the query's own signs; after all C(K,G) profiles the
 *     sign-flipped cones follow (h flips ascending, profile order, flip
 *     subsets lexicographic over the members sorted by |y| ascending).
 *   - the coordinates of x on basis r are y_i = sum_j R_r[i][j] x_j, each
 *     accumulated in fp32 by fused multiply-adds in order j = 0, 1, ...
 *     (the rotated coordinates only decide integers -- keys and query
 *     orders -- so both sides compute them in the same fp32 order); a
 *     projection on m < d components (the PCA front-end of Sec. 4-B) keeps
 *     the first m rows of the basis and subtracts an offset c_i (the
 *     projected mean) in one final fp32 subtraction; distances always use the
 *     original vectors.
 *   - when N_C is too large for a direct table (the "second-level hash
 *     table" of Sec. 4), the cone id is the same number rank(S) * 2^G +
 *     sign code held in 128 bits; only the occupied cones are stored, in
 *     ascending id order, and a probed cone that holds no point is skipped
 *     (it still counts against the budget C).
 *   - ROSANNA+ (Sec. 4-B): the k-means centroids are an input (clustered
 *     off line); a point belongs to its nearest centroid and is hashed by
 *     its residual x - c (fp32 subtraction); the cone id inside the
 *     composite table is cluster * N_C + cone id of the residual; a query
 *     visits its M nearest clusters (nearest first), in each the first
 *     min(C, N_C) cones of its residual y - c.  "Nearest" is the plain
 *     definition: the smallest squared distance (Eq. 1) in double precision,
 *     ties to the lower centroid index.  A caller that holds another
 *     program's assignment (a GPU that decided a near-tie in fp32 the other
 *     way) may pass it in, and the keys and the search then follow it.
 *   - the ORDERED key (an option beside the paper's set key): the profile is
 *     the tuple (i_1, ..., i_G) of the G largest-magnitude components in
 *     decreasing magnitude (ties to the lower index), numbered in
 *     lexicographic order of the tuples, rank = sum_j c_j (K-1-j)!/(K-G)!
 *     with c_j = i_(j+1) minus the number of earlier members below it; the
 *     sign code puts the largest member (position 1) in the most
 *     significant bit; N_C = K!/(K-G)! 2^G.  Its probe order uses the tree
 *     of ordered prefixes: distance delta = G - (length of the common
 *     ordered prefix with the query's tuple); a profile at distance delta
 *     keeps (i_1..i_(G-delta)), its next member is any component but
 *     i_(G-delta+1) outside the prefix, the later ones any unused component;
 *     inside a class, lexicographic in the members' magnitude ranks; then
 *     the sign-flipped cones as for the set key.
 * Parity pinned by: Fig. 2 worked example, N_C closed forms of Sec. 2,
 * class sizes of Sec. 3-B, invariants and brute-force identities (tests).
 * The intra-class probe order and the sign-flip extension are this
 * project's specification: parity unpinned by the paper for those two parts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_D 1024
#define ORACLE_MAX_L 32

/* Binomial coefficient C(n, k), exact, saturating at UINT64_MAX.  Plain
 * multiplicative formula; every intermediate quotient is an integer. */
uint64_t oracle_binom(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 r = 1;
    for (int64_t i = 1; i <= k; ++i) {
        r = r * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
        if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
    }
    return (uint64_t)r;
}

typedef unsigned __int128 u128;
#define U128_MAX (~(u128)0)

/* C(n, k) in 128 bits, exact, saturating at the 128-bit maximum. */
static u128 binom_wide(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    u128 r = 1;
    for (int64_t i = 1; i <= k; ++i) {
        u128 f = (u128)(n - k + i);
        if (r > U128_MAX / f) return U128_MAX;
        r = r * f / (u128)i;
    }
    return r;
}

/* N_C = C(K, G) * 2^G in 128 bits (lo, hi words).  Returns -1 (and writes
 * nothing) when N_C >= 2^127. */
int oracle_num_cones_wide(int d, int L, uint64_t *lohi)
{
    if (d < 1 || L < 1 || L > d || L > ORACLE_MAX_L || d > ORACLE_MAX_D) return -1;
    u128 c = binom_wide(d, L);
    if (c == U128_MAX || c > (((u128)1 << 127) - 1) >> L) return -1;
    u128 nc = c << L;
    lohi[0] = (uint64_t)nc;
    lohi[1] = (uint64_t)(nc >> 64);
    return 0;
}

/* Number of cones N_C = C(K, G) * 2^G (Sec. 2, Table I).  -1 if it does not
 * fit in 63 bits. */
int64_t oracle_num_cones(int d, int L)
{
    if (d < 1 || L < 1 || L > d || L > 62) return -1;
    uint64_t c = oracle_binom(d, L);
    if (c == UINT64_MAX || c > ((uint64_t)INT64_MAX >> L)) return -1;
    return (int64_t)(c << L);
}

/* Indices of the components of y sorted by decreasing magnitude,
 * i_1, i_2, ..., i_K of Sec. 3-B.  Selection sort: at each position take the
 * not-yet-used index with the largest |y|, the lowest index on ties. */
void oracle_magnitude_order(const float *y, int d, int32_t *order)
{
    unsigned char used[ORACLE_MAX_D];
    memset(used, 0, (size_t)d);
    for (int pos = 0; pos < d; ++pos) {
        int best = -1;
        for (int j = 0; j < d; ++j) {
            if (used[j]) continue;
            if (best < 0 || fabsf(y[j]) > fabsf(y[best])) best = j;
        }
        used[best] = 1;
        order[pos] = best;
    }
}

/* Cone id of the profile S (G distinct component indices, any order) with the
 * signs of y on its members, optionally with the members listed in
 * flip_mask (bit m set = flip the sign of the member whose position in the
 * ascending-|y| ordering of S is m) sign-inverted. */
static u128 cone_of_profile_wide(const int32_t *S_in, int L, const float *y,
                                 const int32_t *rank_of, uint32_t flip_mask)
{
    int32_t s[ORACLE_MAX_L];
    memcpy(s, S_in, sizeof(int32_t) * (size_t)L);
    /* sort S by component index, ascending (insertion sort) */
    for (int a = 1; a < L; ++a) {
        int32_t v = s[a];
        int b = a - 1;
        while (b >= 0 && s[b] > v) { s[b + 1] = s[b]; --b; }
        s[b + 1] = v;
    }
    u128 rank = 0;
    for (int j = 0; j < L; ++j) rank += binom_wide(s[j], j + 1);
    u128 code = 0;
    for (int j = 0; j < L; ++j) {
        uint32_t bit = (y[s[j]] >= 0.0f) ? 1u : 0u;
        if (flip_mask) {
            /* position of s[j] in S sorted by |y| ascending = number of members
             * with a larger rank (smaller magnitude) than s[j] */
            int pos = 0;
            for (int t = 0; t < L; ++t)
                if (rank_of[s[t]] > rank_of[s[j]]) ++pos;
            if ((flip_mask >> pos) & 1u) bit ^= 1u;
        }
        code |= (u128)bit << (L - 1 - j);
    }
    return (rank << L) | code;
}

/* The same id when N_C < 2^31 (a direct table). */
static uint32_t cone_of_profile(const int32_t *S_in, int L, const float *y,
                                const int32_t *rank_of, uint32_t flip_mask)
{
    return (uint32_t)cone_of_profile_wide(S_in, L, y, rank_of, flip_mask);
}

/* Cone id of one vector (Sec. 2): profile = the G largest-magnitude
 * components (as an unordered set), cone = profile plus their signs. */
uint32_t oracle_key(const float *x, int d, int L)
{
    int32_t order[ORACLE_MAX_D];
    oracle_magnitude_order(x, d, order);
    return cone_of_profile(order, L, x, NULL, 0);
}

void oracle_keys(const float *X, int64_t N, int d, int L, uint32_t *keys)
{
    for (int64_t n = 0; n < N; ++n) keys[n] = oracle_key(X + n * d, d, L);
}

/* 128-bit cone ids of N vectors, two words (low, high) per vector. */
void oracle_keys_wide(const float *X, int64_t N, int d, int L, uint64_t *keys)
{
    int32_t order[ORACLE_MAX_D];
    for (int64_t n = 0; n < N; ++n) {
        oracle_magnitude_order(X + n * d, d, order);
        u128 k = cone_of_profile_wide(order, L, X + n * d, NULL, 0);
        keys[2 * n] = (uint64_t)k;
        keys[2 * n + 1] = (uint64_t)(k >> 64);
    }
}

/* ---------------------------------------------------------------- ORDERED key */

/* (K - 1 - j)! / (K - G)!: the number of ways to fill the tuple positions
 * after position j (0-based) with distinct unused components. */
static uint64_t falling_after(int d, int L, int j)
{
    uint64_t f = 1;
    for (int m = j + 1; m < L; ++m) {
        uint64_t v = (uint64_t)(d - m);
        if (f > UINT64_MAX / v) return UINT64_MAX;
        f *= v;
    }
    return f;
}

/* N_C of the ORDERED key: K!/(K-G)! * 2^G; -1 if it does not fit in 63 bits. */
int64_t oracle_num_cones_ordered(int d, int L)
{
    if (d < 1 || L < 1 || L > d || L > 62) return -1;
    uint64_t f = falling_after(d, L, -1);
    if (f == UINT64_MAX || f > ((uint64_t)INT64_MAX >> L)) return -1;
    return (int64_t)(f << L);
}

/* Cone id of the ordered profile T (G distinct components in tuple order)
 * with the signs of y on its members, the members whose position in the
 * ascending-|y| ordering of T is set in flip_mask sign-inverted. */
static uint32_t ordered_cone(const int32_t *T, int d, int L, const float *y, const int32_t *rank_of,
                             uint32_t flip_mask)
{
    uint64_t rank = 0;
    for (int j = 0; j < L; ++j) {
        int below = 0;
        for (int t = 0; t < j; ++t)
            if (T[t] < T[j]) ++below;
        rank += (uint64_t)(T[j] - below) * falling_after(d, L, j);
    }
    uint32_t code = 0;
    for (int j = 0; j < L; ++j) {
        uint32_t bit = (y[T[j]] >= 0.0f) ? 1u : 0u;
        if (flip_mask) {
            int pos = 0;
            for (int t = 0; t < L; ++t)
                if (rank_of[T[t]] > rank_of[T[j]]) ++pos;
            if ((flip_mask >> pos) & 1u) bit ^= 1u;
        }
        code |= bit << (L - 1 - j);
    }
    return (uint32_t)((rank << L) | code);
}

/* ORDERED cone id of one vector: its G largest-magnitude components in
 * decreasing magnitude, with their signs. */
uint32_t oracle_key_ordered(const float *x, int d, int L)
{
    int32_t order[ORACLE_MAX_D];
    oracle_magnitude_order(x, d, order);
    return ordered_cone(order, d, L, x, NULL, 0);
}

void oracle_keys_ordered(const float *X, int64_t N, int d, int L, uint32_t *keys)
{
    for (int64_t n = 0; n < N; ++n) keys[n] = oracle_key_ordered(X + n * d, d, L);
}

/* Bucket index: offsets[N_C + 1] (exclusive prefix sum of the cone counts)
 * and perm[N] (point ids, ascending inside each cone: a stable counting
 * sort).  The paper only says that one hash table per basis maps cones to
 * points (Sec. 4, preparation phase). */
void oracle_buckets(const uint32_t *keys, int64_t N, int64_t NC,
                    uint32_t *offsets, uint32_t *perm)
{
    for (int64_t c = 0; c <= NC; ++c) offsets[c] = 0;
    for (int64_t n = 0; n < N; ++n) offsets[keys[n] + 1] += 1;
    for (int64_t c = 0; c < NC; ++c) offsets[c + 1] += offsets[c];
    uint32_t *cursor = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(NC + 1));
    memcpy(cursor, offsets, sizeof(uint32_t) * (size_t)(NC + 1));
    for (int64_t n = 0; n < N; ++n) perm[cursor[keys[n]]++] = (uint32_t)n;
    free(cursor);
}

/* Second-level table for large N_C (Sec. 4 keeps a further hash level for
 * cone counts too large for a direct table): only occupied cones are kept.  perm[N] lists the point ids sorted by (128-bit cone id, id);
 * uniq[2 * n_occ] holds the distinct ids in ascending order (low, high
 * words) and offsets[n_occ + 1] the start of each one's points in perm.
 * Returns n_occ.  The sort is the C library's qsort on (cone id, point id)
 * pairs. */
struct wide_pair {
    u128 key;
    uint32_t id;
};

static int cmp_wide_pair(const void *a, const void *b)
{
    const struct wide_pair *x = (const struct wide_pair *)a, *y = (const struct wide_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

static u128 wide_at(const uint64_t *w, int64_t i) { return ((u128)w[2 * i + 1] << 64) | w[2 * i]; }

int64_t oracle_buckets_wide(const uint64_t *keys, int64_t N, uint32_t *perm, uint64_t *uniq, uint32_t *offsets)
{
    struct wide_pair *v = (struct wide_pair *)malloc(sizeof(struct wide_pair) * (size_t)(N > 0 ? N : 1));
    for (int64_t n = 0; n < N; ++n) {
        v[n].key = wide_at(keys, n);
        v[n].id = (uint32_t)n;
    }
    qsort(v, (size_t)N, sizeof(struct wide_pair), cmp_wide_pair);
    int64_t n_occ = 0;
    for (int64_t i = 0; i < N; ++i) {
        perm[i] = v[i].id;
        if (i == 0 || v[i].key != v[i - 1].key) {
            uniq[2 * n_occ] = (uint64_t)v[i].key;
            uniq[2 * n_occ + 1] = (uint64_t)(v[i].key >> 64);
            offsets[n_occ] = (uint32_t)i;
            ++n_occ;
        }
    }
    offsets[n_occ] = (uint32_t)N;
    free(v);
    return n_occ;
}

/* Position of cone id key among the n_occ ascending ids of uniq, or -1 if
 * no point lies in that cone (binary search). */
static int64_t find_cone(const uint64_t *uniq, int64_t n_occ, u128 key)
{
    int64_t lo = 0, hi = n_occ;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (wide_at(uniq, mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n_occ && wide_at(uniq, lo) == key) ? lo : -1;
}

/* Advance comb[0..m-1] (strictly increasing values in [lo, hi]) to the next
 * combination in lexicographic order.  Returns 0 when exhausted. */
static int next_combination(int32_t *comb, int m, int lo, int hi)
{
    (void)lo;
    int i = m - 1;
    while (i >= 0 && comb[i] == hi - (m - 1 - i)) --i;
    if (i < 0) return 0;
    comb[i] += 1;
    for (int j = i + 1; j < m; ++j) comb[j] = comb[j - 1] + 1;
    return 1;
}

/* Enumerate the level-G profiles in the paper's neighbouring-cone order
 * (Sec. 3-B): distance delta = G - (level of the closest common ancestor
 * with the query's profile) ascending; the profiles at distance delta keep
 * the query's top G-delta components and take the other delta members from
 * the ranks G-delta+2 .. K (rank G-delta+1 excluded, otherwise the common
 * ancestor would be deeper); inside a class, lexicographic in those ranks.
 * Calls emit(S) for each profile until it returns nonzero.  Ranks are
 * 1-based in the paper; positions into order[] here are 0-based. */
typedef int (*profile_cb)(const int32_t *S, void *ctx);

static void enumerate_profiles(const int32_t *order, int d, int L,
                               profile_cb emit, void *ctx)
{
    int32_t S[ORACLE_MAX_L];
    int32_t T[ORACLE_MAX_L];
    for (int delta = 0; delta <= L; ++delta) {
        int keep = L - delta;
        for (int j = 0; j < keep; ++j) S[j] = order[j];
        if (delta == 0) {
            if (emit(S, ctx)) return;
            continue;
        }
        /* 0-based positions keep+1 .. d-1 (rank keep+1 is position keep) */
        int lo = keep + 1, hi = d - 1;
        if (hi - lo + 1 < delta) continue;
        for (int j = 0; j < delta; ++j) T[j] = lo + j;
        do {
            for (int j = 0; j < delta; ++j) S[keep + j] = order[T[j]];
            if (emit(S, ctx)) return;
        } while (next_combination(T, delta, lo, hi));
    }
}

struct probe_ctx {
    const float *y;
    const int32_t *rank_of;
    int L;
    int64_t P, count;
    uint32_t *out;      /* direct-table ids, or */
    uint64_t *out_wide; /* 128-bit ids, two words each */
    uint32_t flip_mask; /* 0 in the first sweep */
    int h;              /* flips per cone in the current sweep */
    int32_t F[ORACLE_MAX_L];
};

static void emit_cone(struct probe_ctx *c, const int32_t *S, uint32_t mask)
{
    u128 k = cone_of_profile_wide(S, c->L, c->y, c->rank_of, mask);
    if (c->out) {
        c->out[c->count] = (uint32_t)k;
    } else {
        c->out_wide[2 * c->count] = (uint64_t)k;
        c->out_wide[2 * c->count + 1] = (uint64_t)(k >> 64);
    }
    c->count++;
}

static int emit_unflipped(const int32_t *S, void *vctx)
{
    struct probe_ctx *c = (struct probe_ctx *)vctx;
    if (c->count >= c->P) return 1;
    emit_cone(c, S, 0);
    return c->count >= c->P;
}

static int emit_flipped(const int32_t *S, void *vctx)
{
    struct probe_ctx *c = (struct probe_ctx *)vctx;
    int32_t F[ORACLE_MAX_L];
    for (int j = 0; j < c->h; ++j) F[j] = j;
    do {
        if (c->count >= c->P) return 1;
        uint32_t mask = 0;
        for (int j = 0; j < c->h; ++j) mask |= 1u << F[j];
        emit_cone(c, S, mask);
    } while (next_combination(F, c->h, 0, c->L - 1));
    return c->count >= c->P;
}

/* Ordered list of cones to visit for query y (Algorithm 1, "find ordered
 * list of cones"), truncated at P entries.  Returns the number written,
 * min(P, N_C). */
static int64_t probes_into(const float *y, int d, int L, int64_t P, uint32_t *out, uint64_t *out_wide)
{
    int32_t order[ORACLE_MAX_D], rank_of[ORACLE_MAX_D];
    oracle_magnitude_order(y, d, order);
    for (int r = 0; r < d; ++r) rank_of[order[r]] = r;
    struct probe_ctx c;
    c.y = y; c.rank_of = rank_of; c.L = L; c.P = P; c.count = 0; c.out = out; c.out_wide = out_wide;
    c.flip_mask = 0; c.h = 0;
    enumerate_profiles(order, d, L, emit_unflipped, &c);
    for (int h = 1; h <= L && c.count < P; ++h) {
        c.h = h;
        enumerate_profiles(order, d, L, emit_flipped, &c);
    }
    return c.count;
}

int64_t oracle_probes(const float *y, int d, int L, int64_t P, uint32_t *out)
{
    return probes_into(y, d, L, P, out, NULL);
}

/* The same list with 128-bit ids (two words each), for N_C of any size. */
int64_t oracle_probes_wide(const float *y, int d, int L, int64_t P, uint64_t *out)
{
    return probes_into(y, d, L, P, NULL, out);
}

/* The ordered profiles in their probe order (see the header): class delta
 * = 0..G; in class delta the prefix (i_1..i_(G-delta)) and delta more
 * members at magnitude ranks (0-based positions into order[]) p_1 ..
 * p_delta, p_1 in keep+1 .. K-1, the later ones in keep .. K-1, all
 * distinct, the rank tuple in lexicographic order (nested ascending loops,
 * written as an odometer).  Calls emit(T) until it returns nonzero. */
static void enumerate_ordered_profiles(const int32_t *order, int d, int L, profile_cb emit, void *ctx)
{
    int32_t T[ORACLE_MAX_L], p[ORACLE_MAX_L];
    for (int delta = 0; delta <= L; ++delta) {
        const int keep = L - delta;
        for (int j = 0; j < keep; ++j) T[j] = order[j];
        if (delta == 0) {
            if (emit(T, ctx)) return;
            continue;
        }
        if (keep + 1 > d - 1) continue;
        /* odometer over (p_1, ..., p_delta): position m takes the smallest
         * admissible value above its current one, unused by positions < m */
        int m = 0;
        p[0] = keep;  /* incremented to keep + 1 below */
        for (;;) {
            /* advance position m */
            int v = p[m] + 1;
            for (;; ++v) {
                int used = 0;
                for (int t = 0; t < m; ++t)
                    if (p[t] == v) used = 1;
                if (!used) break;
            }
            if (v > d - 1) {
                if (m == 0) break;
                --m;
                continue;
            }
            p[m] = v;
            if (m + 1 < delta) {
                ++m;
                p[m] = keep - 1;  /* the smallest value of a later position is keep */
                continue;
            }
            for (int j = 0; j < delta; ++j) T[keep + j] = order[p[j]];
            if (emit(T, ctx)) return;
        }
    }
}

struct oprobe_ctx {
    const float *y;
    const int32_t *rank_of;
    int d, L, h;
    int64_t P, count;
    uint32_t *out;
};

static int emit_ordered_unflipped(const int32_t *T, void *vctx)
{
    struct oprobe_ctx *c = (struct oprobe_ctx *)vctx;
    if (c->count >= c->P) return 1;
    c->out[c->count++] = ordered_cone(T, c->d, c->L, c->y, c->rank_of, 0);
    return c->count >= c->P;
}

static int emit_ordered_flipped(const int32_t *T, void *vctx)
{
    struct oprobe_ctx *c = (struct oprobe_ctx *)vctx;
    int32_t F[ORACLE_MAX_L];
    for (int j = 0; j < c->h; ++j) F[j] = j;
    do {
        if (c->count >= c->P) return 1;
        uint32_t mask = 0;
        for (int j = 0; j < c->h; ++j) mask |= 1u << F[j];
        c->out[c->count++] = ordered_cone(T, c->d, c->L, c->y, c->rank_of, mask);
    } while (next_combination(F, c->h, 0, c->L - 1));
    return c->count >= c->P;
}

/* The ordered cone list of the ORDERED key, truncated at P entries; returns
 * min(P, N_C). */
int64_t oracle_probes_ordered(const float *y, int d, int L, int64_t P, uint32_t *out)
{
    int32_t order[ORACLE_MAX_D], rank_of[ORACLE_MAX_D];
    oracle_magnitude_order(y, d, order);
    for (int r = 0; r < d; ++r) rank_of[order[r]] = r;
    struct oprobe_ctx c;
    c.y = y; c.rank_of = rank_of; c.d = d; c.L = L; c.h = 0; c.P = P; c.count = 0; c.out = out;
    enumerate_ordered_profiles(order, d, L, emit_ordered_unflipped, &c);
    for (int h = 1; h <= L && c.count < P; ++h) {
        c.h = h;
        enumerate_ordered_profiles(order, d, L, emit_ordered_flipped, &c);
    }
    return c.count;
}

/* Candidate exclusion used by the patch workload: data id n sits at grid
 * position (n / grid_w, n % grid_w); it is skipped for a query taken from
 * grid id src when the Chebyshev distance is <= radius. */
static int excluded(int64_t n, int64_t src, int64_t grid_w, int64_t radius)
{
    if (src < 0 || grid_w <= 0) return 0;
    int64_t dr = n / grid_w - src / grid_w;
    int64_t dc = n % grid_w - src % grid_w;
    if (dr < 0) dr = -dr;
    if (dc < 0) dc = -dc;
    return (dr > dc ? dr : dc) <= radius;
}

/* Squared Euclidean distance in double precision (Eq. 1). */
static double sqdist(const float *x, const float *y, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = (double)x[i] - (double)y[i];
        s += t * t;
    }
    return s;
}

/* Keep the k best (distance, id) pairs, ascending by distance then id. */
static void topk_insert(double *bd, int64_t *bi, int k, double dist, int64_t id)
{
    if (dist > bd[k - 1] || (dist == bd[k - 1] && id >= bi[k - 1])) return;
    int j = k - 1;
    while (j > 0 && (bd[j - 1] > dist || (bd[j - 1] == dist && bi[j - 1] > id))) {
        bd[j] = bd[j - 1];
        bi[j] = bi[j - 1];
        --j;
    }
    bd[j] = dist;
    bi[j] = id;
}

static void topk_init(double *bd, int64_t *bi, int k)
{
    for (int j = 0; j < k; ++j) { bd[j] = INFINITY; bi[j] = -1; }
}

/* ROSANNA search with one basis (Algorithm 1 with R = 1): hash the query,
 * build its ordered cone list, and scan the cones' points in that order with
 * exact distances, keeping the k nearest.  With R = 1 the visited cones are
 * disjoint, so the "analyzed" flag of Algorithm 1 never fires and partial
 * distance elimination only skips work, never changes the result; both are
 * left out.  query_src may be NULL (no exclusion).  Outputs ids[Q*k] (-1 pad)
 * and dists[Q*k] (+inf pad), squared distances.  probe_buf must hold P
 * entries.  cand_count (may be NULL) receives the number of candidates
 * scanned per query. */
void oracle_search_mode(const float *X, int64_t N, int d, int L, int key_mode,
                        const uint32_t *offsets, const uint32_t *perm,
                        const float *Y, int64_t Q, int64_t P, int k,
                        const int64_t *query_src, int64_t grid_w, int64_t radius,
                        int64_t *ids, double *dists, int64_t *cand_count);

void oracle_search(const float *X, int64_t N, int d, int L,
                   const uint32_t *offsets, const uint32_t *perm,
                   const float *Y, int64_t Q, int64_t P, int k,
                   const int64_t *query_src, int64_t grid_w, int64_t radius,
                   int64_t *ids, double *dists, int64_t *cand_count)
{
    oracle_search_mode(X, N, d, L, 0, offsets, perm, Y, Q, P, k, query_src, grid_w, radius, ids, dists,
                       cand_count);
}

/* As oracle_search, for the set key (key_mode 0) or the ORDERED key (1). */
void oracle_search_mode(const float *X, int64_t N, int d, int L, int key_mode,
                        const uint32_t *offsets, const uint32_t *perm,
                        const float *Y, int64_t Q, int64_t P, int k,
                        const int64_t *query_src, int64_t grid_w, int64_t radius,
                        int64_t *ids, double *dists, int64_t *cand_count)
{
    (void)N;
    int64_t NC = key_mode ? oracle_num_cones_ordered(d, L) : oracle_num_cones(d, L);
    if (P > NC) P = NC;
    uint32_t *probes = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P > 0 ? P : 1));
    for (int64_t q = 0; q < Q; ++q) {
        const float *y = Y + q * d;
        double *bd = dists + q * k;
        int64_t *bi = ids + q * k;
        topk_init(bd, bi, k);
        int64_t np = key_mode ? oracle_probes_ordered(y, d, L, P, probes) : oracle_probes(y, d, L, P, probes);
        int64_t cands = 0;
        int64_t src = query_src ? query_src[q] : -1;
        for (int64_t l = 0; l < np; ++l) {
            uint32_t c = probes[l];
            for (uint32_t r = offsets[c]; r < offsets[c + 1]; ++r) {
                int64_t n = perm[r];
                if (excluded(n, src, grid_w, radius)) continue;
                ++cands;
                topk_insert(bd, bi, k, sqdist(X + n * d, y, d), n);
            }
        }
        if (cand_count) cand_count[q] = cands;
    }
    free(probes);
}

/* The search of oracle_search over the second-level table of
 * oracle_buckets_wide: the same ordered cone list with 128-bit ids, each
 * looked up among the occupied cones; P is clamped to N_C (128-bit). */
void oracle_search_wide(const float *X, int64_t N, int d, int L, int64_t n_occ,
                        const uint64_t *uniq, const uint32_t *offsets, const uint32_t *perm,
                        const float *Y, int64_t Q, int64_t P, int k,
                        const int64_t *query_src, int64_t grid_w, int64_t radius,
                        int64_t *ids, double *dists, int64_t *cand_count)
{
    (void)N;
    uint64_t nc[2];
    if (oracle_num_cones_wide(d, L, nc) != 0) return;
    u128 NC = ((u128)nc[1] << 64) | nc[0];
    if ((u128)P > NC) P = (int64_t)NC;
    uint64_t *probes = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)(P > 0 ? P : 1));
    for (int64_t q = 0; q < Q; ++q) {
        const float *y = Y + q * d;
        double *bd = dists + q * k;
        int64_t *bi = ids + q * k;
        topk_init(bd, bi, k);
        int64_t np = oracle_probes_wide(y, d, L, P, probes);
        int64_t cands = 0;
        int64_t src = query_src ? query_src[q] : -1;
        for (int64_t l = 0; l < np; ++l) {
            int64_t c = find_cone(uniq, n_occ, wide_at(probes, l));
            if (c < 0) continue;
            for (uint32_t r = offsets[c]; r < offsets[c + 1]; ++r) {
                int64_t n = perm[r];
                if (excluded(n, src, grid_w, radius)) continue;
                ++cands;
                topk_insert(bd, bi, k, sqdist(X + n * d, y, d), n);
            }
        }
        if (cand_count) cand_count[q] = cands;
    }
    free(probes);
}

/* ---------------------------------------------------------------- ROSANNA+ */

/* The M nearest of K centroids (K x d) of each of n vectors, nearest first,
 * by (squared distance in double precision, centroid index): out[i * M + j];
 * -1 pads when M > K. */
void oracle_nearest_centroids(const float *X, int64_t n, int d, const float *C, int K, int M, int32_t *out)
{
    double *bd = (double *)malloc(sizeof(double) * (size_t)M);
    int64_t *bi = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);
    for (int64_t i = 0; i < n; ++i) {
        topk_init(bd, bi, M);
        for (int c = 0; c < K; ++c) topk_insert(bd, bi, M, sqdist(X + i * d, C + (int64_t)c * d, d), c);
        for (int j = 0; j < M; ++j) out[i * M + j] = (int32_t)bi[j];
    }
    free(bd);
    free(bi);
}

/* Composite 128-bit cone ids of ROSANNA+ (two words per point) and the
 * cluster of each point: asg[n] = nearest centroid, residual r = x - c in
 * fp32, id = asg * N_C + cone id of r.  asg_in (may be NULL) gives the
 * assignment instead of the nearest centroid (copied to asg).  Returns -1 if
 * K * N_C >= 2^127 or an entry of asg_in is not a centroid. */
int oracle_keys_clustered(const float *X, int64_t N, int d, int L, const float *C, int K, uint64_t *keys,
                          int32_t *asg, const int32_t *asg_in)
{
    uint64_t nc[2];
    if (oracle_num_cones_wide(d, L, nc) != 0) return -1;
    u128 NC = ((u128)nc[1] << 64) | nc[0];
    if ((u128)K > (((u128)1 << 127) - 1) / NC) return -1;
    float *r = (float *)malloc(sizeof(float) * (size_t)d);
    int32_t order[ORACLE_MAX_D];
    if (asg_in) {
        for (int64_t n = 0; n < N; ++n) {
            if (asg_in[n] < 0 || asg_in[n] >= K) { free(r); return -1; }
            asg[n] = asg_in[n];
        }
    } else {
        oracle_nearest_centroids(X, N, d, C, K, 1, asg);
    }
    for (int64_t n = 0; n < N; ++n) {
        const float *c = C + (int64_t)asg[n] * d;
        for (int i = 0; i < d; ++i) r[i] = X[n * d + i] - c[i];
        oracle_magnitude_order(r, d, order);
        u128 k = (u128)asg[n] * NC + cone_of_profile_wide(order, L, r, NULL, 0);
        keys[2 * n] = (uint64_t)k;
        keys[2 * n + 1] = (uint64_t)(k >> 64);
    }
    free(r);
    return 0;
}

/* ROSANNA+ search over the composite table of oracle_buckets_wide (keys of
 * oracle_keys_clustered): for each of the query's M nearest clusters,
 * nearest first, the first min(P, N_C) cones of the residual y - c,
 * looked up among the occupied composite ids; exact top-k over the
 * candidates (the clusters are disjoint, so no point is seen twice).
 * near_in (may be NULL) gives each query's M clusters (Q x M, -1 entries
 * skipped) instead of its M nearest. */
void oracle_search_clustered(const float *X, int64_t N, int d, int L, const float *C, int K, int M,
                             int64_t n_occ, const uint64_t *uniq, const uint32_t *offsets, const uint32_t *perm,
                             const float *Y, int64_t Q, int64_t P, int k, int64_t *ids, double *dists,
                             int64_t *cand_count, const int32_t *near_in)
{
    (void)N;
    (void)K;
    uint64_t nc[2];
    if (oracle_num_cones_wide(d, L, nc) != 0) return;
    u128 NC = ((u128)nc[1] << 64) | nc[0];
    if ((u128)P > NC) P = (int64_t)NC;
    uint64_t *probes = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)(P > 0 ? P : 1));
    int32_t *near = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    float *r = (float *)malloc(sizeof(float) * (size_t)d);
    for (int64_t q = 0; q < Q; ++q) {
        const float *y = Y + q * d;
        double *bd = dists + q * k;
        int64_t *bi = ids + q * k;
        topk_init(bd, bi, k);
        if (near_in) memcpy(near, near_in + q * M, sizeof(int32_t) * (size_t)M);
        else oracle_nearest_centroids(y, 1, d, C, K, M, near);
        int64_t cands = 0;
        for (int j = 0; j < M; ++j) {
            if (near[j] < 0) continue;
            const float *c = C + (int64_t)near[j] * d;
            for (int i = 0; i < d; ++i) r[i] = y[i] - c[i];
            int64_t np = oracle_probes_wide(r, d, L, P, probes);
            for (int64_t l = 0; l < np; ++l) {
                int64_t cc = find_cone(uniq, n_occ, (u128)near[j] * NC + wide_at(probes, l));
                if (cc < 0) continue;
                for (uint32_t row = offsets[cc]; row < offsets[cc + 1]; ++row) {
                    int64_t n = perm[row];
                    ++cands;
                    topk_insert(bd, bi, k, sqdist(X + n * d, y, d), n);
                }
            }
        }
        if (cand_count) cand_count[q] = cands;
    }
    free(probes);
    free(near);
    free(r);
}

/* Coordinates on a rotated basis (Sec. 3-D, "projection of y on the r-th
 * basis"): out[i][r] = sum_j Rm[r][j] X[i][j] in fp32, fused multiply-adds in
 * order j = 0..d-1 from 0.  Rm: d x d row-major (row r = basis vector r). */
void oracle_rotate(const float *Rm, const float *X, int64_t n, int d, float *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < d; ++r) {
            float acc = 0.0f;
            for (int j = 0; j < d; ++j) acc = fmaf(Rm[(int64_t)r * d + j], X[i * d + j], acc);
            out[i * d + r] = acc;
        }
}

/* Projection on m <= d components (Sec. 4-B, PCA front-end): out[i][r] =
 * (sum_j Pm[r][j] X[i][j]) - off[r], the sum in fp32 fused multiply-adds in
 * order j = 0..d-1 from 0, then one fp32 subtraction (off may be NULL: no
 * offset).  Pm: m x d row-major. */
void oracle_project(const float *Pm, const float *off, const float *X, int64_t n, int d, int m, float *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < m; ++r) {
            float acc = 0.0f;
            for (int j = 0; j < d; ++j) acc = fmaf(Pm[(int64_t)r * d + j], X[i * d + j], acc);
            out[i * m + r] = off ? acc - off[r] : acc;
        }
}

void oracle_search_multi_proj(const float *X, int64_t N, int d, int L, int R, int m, const float *projs,
                              const float *projoff, const uint32_t *offsets, const uint32_t *perms,
                              const float *Y, int64_t Q, int64_t P, int k, int64_t *ids, double *dists,
                              int64_t *cand_count);

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Search over R bases (Sec. 3-D): basis r has its own cone index
 * (offsets_r, perm_r, built from the data's coordinates on that basis) and
 * its own list of the query's first min(P, N_C) cones, made from the query's
 * coordinates on that basis.  The candidates are the union of the points of
 * all R lists' cones -- a point that falls in probed cones of several bases
 * is one candidate, its distance computed once -- and the answer is the
 * exact top-k (Eq. 1, original vectors) over that union.  rots: R x d x d;
 * offsets: R x (N_C + 1); perms: R x N.  Outputs as oracle_search
 * (cand_count: size of the union). */
void oracle_search_multi(const float *X, int64_t N, int d, int L, int R, const float *rots,
                         const uint32_t *offsets, const uint32_t *perms, const float *Y, int64_t Q,
                         int64_t P, int k, int64_t *ids, double *dists, int64_t *cand_count)
{
    oracle_search_multi_proj(X, N, d, L, R, d, rots, NULL, offsets, perms, Y, Q, P, k, ids, dists, cand_count);
}

/* As oracle_search_multi, on R projections of m components each (m x d
 * matrices projs, offsets projoff R x m or NULL): keys and probes on the m
 * projected coordinates (N_C = C(m, G) 2^G), distances on the d originals. */
void oracle_search_multi_proj(const float *X, int64_t N, int d, int L, int R, int m, const float *projs,
                              const float *projoff, const uint32_t *offsets, const uint32_t *perms,
                              const float *Y, int64_t Q, int64_t P, int k, int64_t *ids, double *dists,
                              int64_t *cand_count)
{
    int64_t NC = oracle_num_cones(m, L);
    if (P > NC) P = NC;
    uint32_t *probes = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P > 0 ? P : 1));
    float *yr = (float *)malloc(sizeof(float) * (size_t)m);
    /* a point can be listed once per basis */
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R * N > 0 ? R * N : 1));
    for (int64_t q = 0; q < Q; ++q) {
        const float *y = Y + q * d;
        double *bd = dists + q * k;
        int64_t *bi = ids + q * k;
        /* 1. the points of every basis's probed cones */
        int64_t nc = 0;
        for (int r = 0; r < R; ++r) {
            oracle_project(projs + (int64_t)r * m * d, projoff ? projoff + (int64_t)r * m : NULL, y, 1, d, m, yr);
            int64_t np = oracle_probes(yr, m, L, P, probes);
            const uint32_t *off = offsets + (int64_t)r * (NC + 1);
            const uint32_t *perm = perms + (int64_t)r * N;
            for (int64_t l = 0; l < np; ++l)
                for (uint32_t row = off[probes[l]]; row < off[probes[l] + 1]; ++row) cand[nc++] = perm[row];
        }
        /* 2. their union: sorted, repeated ids dropped */
        qsort(cand, (size_t)nc, sizeof(int64_t), cmp_i64);
        int64_t nu = 0;
        for (int64_t i = 0; i < nc; ++i)
            if (nu == 0 || cand[nu - 1] != cand[i]) cand[nu++] = cand[i];
        /* 3. exact top-k over the union */
        topk_init(bd, bi, k);
        for (int64_t i = 0; i < nu; ++i) topk_insert(bd, bi, k, sqdist(X + cand[i] * d, y, d), cand[i]);
        if (cand_count) cand_count[q] = nu;
    }
    free(probes);
    free(yr);
    free(cand);
}

/* Exact linear search (Eq. 1): the k nearest of all N points. */
void oracle_bruteforce(const float *X, int64_t N, int d, const float *Y,
                       int64_t Q, int k, const int64_t *query_src,
                       int64_t grid_w, int64_t radius, int64_t *ids,
                       double *dists)
{
    for (int64_t q = 0; q < Q; ++q) {
        const float *y = Y + q * d;
        double *bd = dists + q * k;
        int64_t *bi = ids + q * k;
        topk_init(bd, bi, k);
        int64_t src = query_src ? query_src[q] : -1;
        for (int64_t n = 0; n < N; ++n) {
            if (excluded(n, src, grid_w, radius)) continue;
            topk_insert(bd, bi, k, sqdist(X + n * d, y, d), n);
        }
    }
}

/* Exact squared distance of given (query, id) pairs, for checking returned
 * distances element by element.  ids < 0 give +inf. */
void oracle_pair_dists(const float *X, int d, const float *Y, int64_t Q,
                       int k, const int64_t *ids, double *out)
{
    for (int64_t q = 0; q < Q; ++q)
        for (int j = 0; j < k; ++j) {
            int64_t n = ids[q * k + j];
            out[q * k + j] = n < 0 ? INFINITY : sqdist(X + n * d, Y + q * d, d);
        }
}
