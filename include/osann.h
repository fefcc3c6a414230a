/*
 * osann.h -- C ABI of libosann: order-statistics cone-hash approximate
 * nearest-neighbour search (Verdoliva, Cozzolino, Poggi, "A reliable
 * order-statistics-based approximate nearest neighbor search algorithm",
 * ROSANNA) on one GB300 GPU (sm_103a), one basis (R = 1).
 *
 * Notation: the paper's K (vector length) is d, G (components used for the
 * hash) is L, C (cones visited per basis) is P, N_C = C(d, L) * 2^L.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device,
 *     caller-owned, contiguous, row-major.  Float inputs must be 16-byte
 *     aligned when d % 4 == 0 (vector loads), otherwise 4-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued on it; only osann_build and
 *     osann_status synchronise it.
 *   - Return value: OSANN_OK (0) or a negative OSANN_ERR_* code;
 *     osann_last_error() then gives a message (thread-local).  On error no
 *     output is guaranteed to be written and no memory is leaked.
 *   - Distances are squared Euclidean distances (Eq. 1) in fp32.  Results
 *     per query are ordered by (distance, id) ascending; missing entries
 *     (fewer than k candidates) are id -1, distance +inf.
 */
#ifndef OSANN_H
#define OSANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OSANN_OK 0
#define OSANN_ERR_INVALID (-1)     /* bad argument (sizes, null pointers, ranges) */
#define OSANN_ERR_UNSUPPORTED (-2) /* N beyond the 31-bit index space (or a size limit below) */
#define OSANN_ERR_OOM (-3)         /* device allocation failed */
#define OSANN_ERR_NONFINITE (-4)   /* NaN or Inf in the data */
#define OSANN_ERR_CUDA (-5)        /* a CUDA call failed */
#define OSANN_ERR_TIMEOUT (-6)     /* a bounded device wait gave up */

/* Search paths (same results, different schedules). */
#define OSANN_PATH_AUTO 0    /* the 16-bit screen when enough queries share a cone (per
                                occupied cone, as counted by a synchronous build), the
                                fp32 tile scan for d > 128, else plain */
#define OSANN_PATH_PLAIN 1   /* one CTA per query scanning its cones */
#define OSANN_PATH_BATCHED 2 /* cone-major work list, persistent fp32 tile scan */
#define OSANN_PATH_BF16 3    /* cone-major work list, bf16 tensor-core screening with a
                                certified error bound, exact fp32 rerank (d <= 128) */
#define OSANN_PATH_FP16 4    /* as OSANN_PATH_BF16 with fp16 operands (data and queries
                                scaled by an exact power of two): an 8x tighter bound,
                                fewer candidates to rerank; the default when batched */

/* Status flags returned by osann_status. */
#define OSANN_STATUS_NONFINITE_DATA 1u
#define OSANN_STATUS_NONFINITE_QUERY 2u
#define OSANN_STATUS_TIMEOUT 4u
#define OSANN_STATUS_BOUND 16u /* a debug check of the screening error bound failed
                                  (only with OSANN_DEBUG_CHECKS=1 in the environment) */

typedef struct osann_index osann_index; /* opaque; owns its device buffers */

/* Optional device allocator used for index buffers and for search
 * workspaces that the caller does not provide.  alloc returns a device
 * pointer (NULL on failure) usable in stream order on `stream`; free
 * releases it in stream order.  Passing NULL functions restores the default
 * (cudaMallocAsync / cudaFreeAsync).  A block always goes back to the
 * allocator that provided it, even after another one is installed (so its
 * functions and ctx must stay valid until the blocks it gave are released).
 * A failed request makes the call return OSANN_ERR_OOM after releasing
 * what it took.  Not thread-safe with concurrent builds. */
typedef void *(*osann_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*osann_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int osann_set_allocator(osann_alloc_fn alloc, osann_free_fn free_fn, void *ctx);

/* Number of cones N_C = C(d, L) * 2^L (Sec. 2, Table I).  Errors:
 * INVALID for d < 1, L < 1, L > d; UNSUPPORTED if N_C >= 2^31. */
int osann_num_cones(int32_t d, int32_t L, int64_t *nc);

/* Cone id of each of n vectors (Sec. 2: profile = unordered set of the L
 * largest-magnitude components, ties to the lower index; cone = profile
 * plus their signs, zero counted positive).  key = rank(S) * 2^L + code with
 * rank(S) = sum_j C(s_j, j+1) over the members in ascending order and
 * code = sum_j [x_{s_j} >= 0] 2^(L-1-j).
 * d_vectors: n x d fp32.  d_keys: n uint32 (written).  1 <= d <= 256,
 * 1 <= L <= min(d, 16).  Non-finite inputs are not reported here. */
int osann_keys(const float *d_vectors, int64_t n, int32_t d, int32_t L, uint32_t *d_keys, void *stream);

/* The same cone ids for any N_C (the numbers of the second-level table,
 * Sec. 4): rank(S) * 2^L + code exact in 128 bits, written as four uint32
 * words per vector, least significant first (d_ids: n x 4, 16-byte
 * aligned).  N_C < 2^100 for every d <= 256, L <= 16. */
int osann_keys_wide(const float *d_vectors, int64_t n, int32_t d, int32_t L, uint32_t *d_ids, void *stream);

/* Magnitude order i_1..i_d of each query (Sec. 3-B): d_order[q*d + r] is the
 * component with the (r+1)-th largest |y| (ties to the lower index), uint8.
 * d_signs[q*8 + w] bit b is set when y[32w + b] >= 0 (8 words per query).
 * 1 <= d <= 256. */
int osann_query_order(const float *d_queries, int64_t Q, int32_t d, uint8_t *d_order, uint32_t *d_signs,
                      void *stream);

/* Build the index of one basis (Sec. 4, preparation phase; Table II):
 * cone keys of all points, cone histogram and exclusive scan (CSR offsets),
 * stable counting sort of point ids by cone, the permuted fp32 copy of the
 * vectors (zero padded to d_pad in {16, 32, 64, 128, 256}) and, for
 * d <= 128, the scaled fp16 operands of the tensor-core screen (the bf16
 * ones are made on the first OSANN_PATH_BF16 search, which then
 * synchronises its stream once).
 * d_data: N x d fp32, read only (the index keeps its own copy).
 * With N_C >= 2^31 the index gets the second-level cone table (see
 * osann_build_ex).  Synchronises `stream` once.  Errors: INVALID (N < 1, d
 * outside [1,256], L outside [1, min(d,16)], out == NULL), UNSUPPORTED
 * (N >= 2^31), NONFINITE (NaN/Inf in d_data), OOM, CUDA. */
int osann_build(const float *d_data, int64_t N, int32_t d, int32_t L, void *stream, osann_index **out);

/* One basis of the multi-basis search (Sec. 3-D, Algorithm 1 with R > 1):
 * as osann_build, but the cone keys -- and, in every later search, the
 * query's magnitude order -- come from the coordinates on the basis d_rot
 * (d x d fp32, row-major, row r = basis vector r, orthonormal; the index
 * keeps a copy): y_r = sum_j d_rot[r][j] x_j, accumulated in fp32 by fused
 * multiply-adds in order j = 0, 1, ... from 0.  Distances still use the
 * original vectors.  d <= 128 (else UNSUPPORTED).  async != 0: as
 * osann_build_async.  The R bases of a search are R such indexes; their
 * per-basis results merge with osann_merge_topk, which drops repeated ids
 * (a point found on several bases is one candidate: the "analyzed" flag of
 * Algorithm 1). */
int osann_build_rot(const float *d_data, int64_t N, int32_t d, int32_t L, const float *d_rot, int32_t async,
                    void *stream, osann_index **out);

/* The PCA front-end of Sec. 4-B (cone keys from the leading principal
 * components, distances on all of them): as osann_build_rot with a projection on m <= d
 * components, d_proj (m x d fp32, row r = axis r) and optional offsets d_off
 * (m fp32, the projected mean; NULL: none): keys and query orders come from
 * y_r = (sum_j d_proj[r][j] x_j) - d_off[r] (fp32 in-order fused
 * multiply-adds, then one subtraction), so N_C = C(m, L) 2^L; distances use
 * all d original components.  1 <= m <= d <= 128. */
int osann_build_proj(const float *d_data, int64_t N, int32_t d, int32_t L, const float *d_proj, const float *d_off,
                     int32_t m, int32_t async, void *stream, osann_index **out);

/* As osann_build, without the final synchronisation (the paper has no
 * counterpart: for pipelines that build and search back to back).  The
 * index is usable at once in stream order on `stream`; its status bits
 * (OSANN_STATUS_NONFINITE_DATA, OSANN_STATUS_TIMEOUT) are left for the next
 * osann_status call, which must be checked before the results are trusted,
 * and max_bucket reads -1 in osann_info until that call. */
int osann_build_async(const float *d_data, int64_t N, int32_t d, int32_t L, void *stream, osann_index **out);

/* Cone table kinds for osann_build_ex.  A direct table holds all N_C cones
 * (CSR offsets over the cone ids) and needs N_C < 2^31.  The second-level
 * table (Sec. 4: an extra hash level for cone counts too large for a
 * direct table) keeps only the occupied cones: the point ids
 * are sorted by 128-bit cone id (osann_keys_wide), the occupied cones are
 * numbered 0..n_occ-1 in ascending id order ("compact" cones), offsets span
 * NC_t = min(N, N_C) + 1 compact cones (those from n_occ on are empty), and
 * a hash table maps a probed id to its compact cone -- or, for an id no
 * point carries, to the empty cone NC_t - 1.  Both kinds give the same
 * search results; AUTO takes the direct table when N_C < 2^31. */
#define OSANN_CONES_AUTO 0
#define OSANN_CONES_DENSE 1
#define OSANN_CONES_HASHED 2

/* Key modes for osann_build_ex.  OSANN_KEY_SET is the paper's profile
 * (Sec. 2: the unordered set of the L largest-magnitude components; the
 * paper does not order the components inside the group).
 * OSANN_KEY_ORDERED keys the tuple (i_1, ..., i_L) of those components in
 * decreasing magnitude (ties: the lower component first) with their
 * signs: N_C = d!/(d-L)! 2^L, id = rank * 2^L + code, rank the tuple's
 * position in lexicographic order, sum_j c_j (d-1-j)!/(d-L)! with c_j =
 * i_(j+1) minus the number of earlier members below it, code bit L-1-j
 * the sign of i_(j+1) (zero positive).  Its probe order follows the tree
 * of ordered prefixes: distance delta = L - (length of the common prefix
 * with the query's tuple); a profile at distance delta keeps
 * (i_1..i_(L-delta)), its next member is any component but i_(L-delta+1)
 * outside the prefix, the later ones any unused component; inside a class
 * lexicographic in the members' magnitude ranks in the query; each with
 * the query's signs, then the sign-flipped cones as for the set key.
 * ORDERED needs N_C < 2^31 (a direct table) and no clusters. */
#define OSANN_KEY_SET 0
#define OSANN_KEY_ORDERED 1

typedef struct {
    const float *d_basis;  /* m x d key basis (osann_build_rot / osann_build_proj), NULL: the identity */
    const float *d_offset; /* m offsets subtracted after projecting, NULL: none (needs d_basis) */
    int32_t m;             /* rows of d_basis (ignored without one) */
    int32_t async;         /* nonzero: no final synchronisation (as osann_build_async) */
    int32_t cone_table;    /* OSANN_CONES_* */
    const float *d_centroids; /* ROSANNA+: K x d k-means centroids (see below), NULL: none */
    int32_t n_clusters;       /* K (0: none) */
    int32_t key_mode;         /* OSANN_KEY_SET (0, the paper's) or OSANN_KEY_ORDERED */
} osann_build_opts;

/* Build with explicit options (opts NULL: as osann_build).  Every other
 * build entry point is this one with the matching options and
 * OSANN_CONES_AUTO.
 * ROSANNA+ (Sec. 4-B: data clustered off line by k-means, a query searching
 * only its nearest clusters): with d_centroids (K x d fp32, read during the
 * build; the index keeps a copy) every point belongs to its nearest centroid
 * c -- by the library's fp32 squared distance (float4 pieces, adjacent-
 * pairwise tree), ties to the lower index -- and is hashed by its residual
 * x - c (fp32); its cone id is cluster * N_C + cone id of the residual, so
 * the table holds K * N_C cones (a second-level table from 2^31 on).
 * Search with osann_search_clusters; osann_search visits the nearest
 * cluster only.  Needs d <= 128, 1 <= K <= 2^24, no key basis.
 * Errors as osann_build, plus: INVALID for a bad cluster set-up,
 * UNSUPPORTED for OSANN_CONES_DENSE with N_C >= 2^31, and for a
 * second-level table of more than 2^30 cones. */
int osann_build_ex(const float *d_data, int64_t N, int32_t d, int32_t L, const osann_build_opts *opts, void *stream,
                   osann_index **out);

/* The cone table of an index.  Any output may be NULL.  hashed: 1 for the
 * second-level table.  n_cones[2]: N_C (low, high 64-bit words).
 * table_cones: cones of the CSR table (the NC of osann_info: N_C, or NC_t).
 * occupied: cones holding at least one point (synchronises `stream`). */
int osann_cones(const osann_index *index, int32_t *hashed, uint64_t *n_cones, int64_t *table_cones,
                int64_t *occupied, void *stream);

/* The 128-bit id of every compact cone of a second-level table: d_ids is
 * table_cones x 4 uint32 words (least significant first); entries past the
 * occupied cones are all ones.  INVALID for a direct table. */
int osann_export_cones(const osann_index *index, uint32_t *d_ids, void *stream);

/* Rebuild an index in place from new data of the same shape (N x d): the
 * build's kernels again (keys, cone table, permuted rows and screening
 * operands; the same basis, centroids and table kind), into the index's own
 * buffers.  Asynchronous, like osann_build_async: the status bits and the
 * largest cone are read by the next osann_status.  The first call allocates
 * the build's temporaries and keeps them with the index; later calls
 * allocate nothing, so a rebuild and searches with caller workspaces can be
 * captured together in a CUDA graph and replayed (searches already in
 * flight on other streams must be complete).  Errors: INVALID, OOM, CUDA. */
int osann_rebuild(osann_index *index, const float *d_data, void *stream);

/* osann_rebuild followed by osann_search on the same stream, with the
 * query-side steps beside the rebuild (as osann_build_search).  With a
 * caller workspace (osann_search_workspace_size of this index) and after one
 * earlier call, it allocates nothing: the whole build-and-search step can be
 * captured in one CUDA graph.  The status bits are left for osann_status. */
int osann_rebuild_search(osann_index *index, const float *d_data, const float *d_queries, int64_t Q, int32_t P,
                         int32_t k, int32_t path, void *d_ws, size_t ws_bytes, int64_t *d_ids, float *d_sqdists,
                         void *stream);

/* Release an index.  NULL is accepted.  The caller must ensure that no
 * work using the index is still pending on any stream. */
int osann_free(osann_index *index);

/* Sizes of an index.  Any output pointer may be NULL.  max_bucket is the
 * largest cone population.  NC is the number of cones of the CSR table:
 * N_C for a direct table, NC_t = min(N, N_C) + 1 for a second-level one
 * (osann_cones gives N_C itself). */
int osann_info(const osann_index *index, int64_t *N, int32_t *d, int32_t *L, int64_t *NC, int64_t *max_bucket);

/* Copy the index's bucket structure out (for verification): d_keys[N]
 * (cone of each point, original order), d_offsets[NC + 1], d_perm[N]
 * (point ids, ascending inside each cone), NC as in osann_info; with a
 * second-level table the cones are the compact ones.  Any pointer may be
 * NULL. */
int osann_export(const osann_index *index, uint32_t *d_keys, uint32_t *d_offsets, uint32_t *d_perm, void *stream);

/* Ordered list of cones to visit (Algorithm 1, "find ordered list of
 * cones"; Sec. 3-B): d_probes[q * P_eff + p], P_eff = min(P, N_C) (with a
 * second-level table: the compact cone of each probed id, NC_t - 1 for an
 * unoccupied one).  Order:
 * profile distance delta = L - (level of the closest common ancestor with
 * the query's profile {i_1..i_L}) ascending; inside a class the substituted
 * ranks in lexicographic order; each profile with the query's signs; then
 * the sign-flipped cones (h flips ascending, profile order, flipped members
 * as h-subsets of the members sorted by |y| ascending).  Needs a workspace of
 * osann_search_workspace_size(index, Q, P, 1, OSANN_PATH_PLAIN) bytes
 * (d_ws may be NULL: then it is allocated and released in stream order). */
int osann_probes(const osann_index *index, const float *d_queries, int64_t Q, int32_t P, uint32_t *d_probes,
                 void *d_ws, size_t ws_bytes, void *stream);

/* Workspace bytes that osann_search / osann_search_excl need for (Q, P, k)
 * on `path`. */
size_t osann_search_workspace_size(const osann_index *index, int64_t Q, int32_t P, int32_t k, int32_t path);

/* ROSANNA+ search (Sec. 4-B) on an index built with centroids: each query
 * visits its M nearest clusters (1 <= M <= 32, clamped to K; nearest first, as in the
 * build), in each the first min(P, N_C) cones of its residual y - c in the
 * order of osann_probes; exact top-k over all their points, as osann_search
 * (same paths, same bits on every path).  Workspace:
 * osann_search_clusters_workspace_size(index, Q, M, P, k, path). */
size_t osann_search_clusters_workspace_size(const osann_index *index, int64_t Q, int32_t M, int32_t P, int32_t k,
                                            int32_t path);
int osann_search_clusters(const osann_index *index, const float *d_queries, int64_t Q, int32_t M, int32_t P,
                          int32_t k, int32_t path, void *d_ws, size_t ws_bytes, int64_t *d_ids, float *d_sqdists,
                          void *stream);

/* Build an index and search it, in one call: the same as osann_build_ex
 * (opts may be NULL) followed by osann_search on the same stream, same
 * results, except that the query-side steps (magnitude orders and probe
 * lists, which do not read the built index) run on a side stream beside the
 * build instead of after it (for a plain direct table; with a basis,
 * centroids or a second-level table they follow the build).  The queries
 * must be ready when the call is made (in stream order).  d_ws may be NULL
 * (allocated and released in stream order); a caller workspace must hold
 * osann_search_workspace_size of the built index.  With opts->async == 0 the
 * call synchronises once at the end and reports the build's status (as
 * osann_build); otherwise the status is left for osann_status.  On success
 * *out is the index (release with osann_free). */
int osann_build_search(const float *d_data, int64_t N, int32_t d, int32_t L, const osann_build_opts *opts,
                       const float *d_queries, int64_t Q, int32_t P, int32_t k, int32_t path, void *d_ws,
                       size_t ws_bytes, int64_t *d_ids, float *d_sqdists, void *stream, osann_index **out);

/* ROSANNA search with one basis (Algorithm 1, R = 1): hash each query,
 * visit its first P_eff = min(P, N_C) cones in the order of osann_probes and
 * return the k nearest candidates by exact squared Euclidean distance
 * (Eq. 1, fp32 direct differences), ordered by (distance, id).  All paths
 * return the same bits: OSANN_PATH_BF16 only screens candidates with a
 * proven error bound before the same fp32 evaluation.
 * d_queries: Q x d fp32.  d_ids: Q x k int64 (point ids, -1 pad).
 * d_sqdists: Q x k fp32 (+inf pad).  d_ws/ws_bytes: workspace of at least
 * osann_search_workspace_size(...) bytes, 256-byte aligned (else
 * OSANN_ERR_INVALID, before anything runs; NULL: allocated and released in
 * stream order).  The same holds for every other call taking d_ws.
 * 1 <= k <= 32, P >= 1, Q >= 0.
 * Asynchronous.  Non-finite queries set OSANN_STATUS_NONFINITE_QUERY (see
 * osann_status); their results are unspecified but in range. */
int osann_search(const osann_index *index, const float *d_queries, int64_t Q, int32_t P, int32_t k, int32_t path,
                 void *d_ws, size_t ws_bytes, int64_t *d_ids, float *d_sqdists, void *stream);

/* As osann_search, with the work list's query group size chosen by the
 * caller (the paper has no counterpart: a tuning knob of the batched
 * paths).  group = 0 takes the default; otherwise it is used when it lies in
 * 1..128 on the tensor-core paths (the MMA tile's query rows) or in
 * 1..128 / max(1, d_pad / 32) on OSANN_PATH_BATCHED, and the default is
 * taken when it does not; the plain path ignores it.  Results are those of
 * osann_search, bit for bit, whatever the group.  The workspace is
 * osann_search_workspace_size_group(...) bytes. */
int osann_search_group(const osann_index *index, const float *d_queries, int64_t Q, int32_t P, int32_t k,
                       int32_t path, int32_t group, void *d_ws, size_t ws_bytes, int64_t *d_ids, float *d_sqdists,
                       void *stream);

/* Layout of the tensor-core screen's query tiles (a tuning knob; the paper
 * has no counterpart).  OSANN_LAYOUT_SMEM: in shared memory beside the cone
 * tiles.  OSANN_LAYOUT_TMEM: in tensor memory beside the accumulators, the
 * MMAs reading only the cone tiles from shared memory (one CTA per SM with
 * more cone-tile stages); possible for d_pad = 128 (64 < d <= 128) without an
 * exclusion radius.  OSANN_LAYOUT_DEFAULT: the library's choice (TMEM where
 * possible). */
#define OSANN_LAYOUT_DEFAULT 0
#define OSANN_LAYOUT_SMEM 1
#define OSANN_LAYOUT_TMEM 2

/* As osann_search_group, with the screen's query-tile layout chosen by the
 * caller (OSANN_LAYOUT_*): ignored off the tensor-core paths, and
 * OSANN_LAYOUT_TMEM takes the default where it is not possible.  Results are
 * those of osann_search, bit for bit, whatever the layout.  The workspace is
 * osann_search_workspace_size_group(...) bytes.  Errors as osann_search; a
 * layout outside 0..2 is OSANN_ERR_INVALID. */
int osann_search_layout(const osann_index *index, const float *d_queries, int64_t Q, int32_t P, int32_t k,
                        int32_t path, int32_t group, int32_t layout, void *d_ws, size_t ws_bytes, int64_t *d_ids,
                        float *d_sqdists, void *stream);
size_t osann_search_workspace_size_group(const osann_index *index, int64_t Q, int32_t P, int32_t k, int32_t path,
                                         int32_t group);

/* As osann_search, skipping for query q every point n whose grid position
 * (n / grid_w, n % grid_w) is within Chebyshev distance `radius` of
 * d_query_src[q]'s position (self and near-duplicates of an image patch).
 * grid_w >= 1, radius >= 0; a negative source disables the filter for
 * that query. */
int osann_search_excl(const osann_index *index, const float *d_queries, const int64_t *d_query_src, int64_t Q,
                      int32_t P, int32_t k, int64_t grid_w, int32_t radius, int32_t path, void *d_ws,
                      size_t ws_bytes, int64_t *d_ids, float *d_sqdists, void *stream);

/* Search without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * at query time -- a plugin inside a host process that owns the device
 * allocator, a latency-critical thread that must not take allocator locks
 * or synchronise, or a program that reserved all device memory up front.
 * It runs the plain path of osann_search (same results, bit for bit) with
 * its scratch in a fixed 32 MiB device array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * Inputs and outputs are as for osann_search; nothing is allocated, freed
 * or returned to an allocator.  The scratch needed is
 * osann_search_workspace_size(index, Q, P, k, OSANN_PATH_PLAIN); calls that
 * need more than 32 MiB fail with OSANN_ERR_INVALID (split the batch), and
 * so do calls made while the current device is not the index's (each device
 * has its own array).
 * The first call on a device looks up the array's device address and the
 * library's per-device tables; make it before any stream capture.  All
 * calls share the one array, which keeps the last call's contents (every
 * byte a call reads it has written first): calls that overlap on the GPU,
 * on any streams, race and must be serialised by the caller. */
int osann_search_noalloc(const osann_index *index, const float *d_queries, int64_t Q, int32_t P, int32_t k,
                         int64_t *d_ids, float *d_sqdists, void *stream);

/* Exact linear search (Eq. 1 over all N points of the index), fp32 direct
 * differences, cuBLAS-free: the ground truth for recall.  d_query_src may
 * be NULL (no exclusion).  Workspace: osann_bruteforce_workspace_size. */
size_t osann_bruteforce_workspace_size(const osann_index *index, int64_t Q, int32_t k);
int osann_bruteforce(const osann_index *index, const float *d_queries, const int64_t *d_query_src, int64_t Q,
                     int32_t k, int64_t grid_w, int32_t radius, void *d_ws, size_t ws_bytes, int64_t *d_ids,
                     float *d_sqdists, void *stream);

/* Counters of the tensor-core screening path since the last call (then
 * cleared), after synchronising `stream`: out4[0] survivors reranked,
 * out4[1] queries whose survivor list overflowed and were rescanned in full,
 * out4[2] / out4[3] error-bound checks made / failed (debug checks only). */
int osann_screen_stats(const osann_index *index, void *stream, int64_t *out4);

/* Synchronise `stream`, return the index's device status flags
 * (OSANN_STATUS_*) accumulated since the last call, and clear them. */
int osann_status(const osann_index *index, void *stream, uint32_t *flags);

/* Message of the last error on this thread ("" if none). */
const char *osann_last_error(void);

/* Instrumentation.  With stats enabled, every stage records CUDA events on
 * its stream; osann_stats_get synchronises those events and returns the
 * accumulated milliseconds and launch count of `stage` (OSANN_STAGE_*).
 * osann_launch_count returns the number of kernels this library has
 * launched in this process. */
#define OSANN_STAGE_DATA_KEYS 0
#define OSANN_STAGE_BUCKETS 1
#define OSANN_STAGE_GATHER 2
#define OSANN_STAGE_QUERY_ORDER 3
#define OSANN_STAGE_PROBES 4
#define OSANN_STAGE_WORKLIST 5
#define OSANN_STAGE_TILE_SCAN 6
#define OSANN_STAGE_MERGE 7
#define OSANN_STAGE_PLAIN_SCAN 8
#define OSANN_STAGE_BRUTEFORCE 9
#define OSANN_STAGE_TC_PREP 10   /* bf16 queries, norms, seed bounds */
#define OSANN_STAGE_TC_SCAN 11   /* tensor-core screening */
#define OSANN_STAGE_TC_RERANK 12 /* exact fp32 rerank of the survivors */
#define OSANN_NUM_STAGES 13
int osann_stats_enable(int on);
int osann_stats_reset(void);
int osann_stats_get(int32_t stage, double *total_ms, int64_t *count);
int64_t osann_launch_count(void);

/* Test hook for failure detection (the paper has no counterpart): the clock
 * budget, in SM cycles, of the plain scan's waits for its staged copies
 * (OSANN_PATH_PLAIN, and the exact rescan of the tensor-core paths).  A wait
 * that runs past it gives up: the kernel lets its copies in flight land
 * (under the full budget), writes what it found for the query at hand and
 * empty results (-1, +inf) for its other queries, and sets
 * OSANN_STATUS_TIMEOUT, which the next osann_status reports; the context
 * stays usable.  0 restores the default of about one second, which no
 * legitimate wait approaches; a budget of a few cycles makes the waits run
 * out.  Process-wide, read at each launch; not for production use.
 * Errors: INVALID for a negative budget. */
int osann_debug_wait_budget(int64_t cycles);

/* Merge of per-shard results (the exchange step of a search sharded by data
 * rows; the paper has no counterpart).  d_ids / d_sqdists hold G lists laid
 * out [G][Q][k] (as osann_search returns them, ids already global, -1 and
 * +inf as padding); the result is the k best of each query's G*k entries by
 * (distance, id), padded with -1 / +inf; an id present in several lists
 * (the same point found on several bases) counts once.  Since keys depend
 * only on a row,
 * the shards' candidate sets partition the unsharded one, and the merge of
 * their k-best lists equals the unsharded search bit for bit.  Ids must be
 * below 2^32 - 1.  1 <= k <= 32.  Asynchronous on `stream`. */
int osann_merge_topk(const int64_t *d_ids, const float *d_sqdists, int32_t G, int64_t Q, int32_t k,
                     int64_t *d_out_ids, float *d_out_sqdists, void *stream);

/* ---------------------------------------------------------------- serving
 *
 * A request server over indexes resident on the device (the paper has no
 * counterpart: this is the serving layer around Algorithm 1).  Requests wait
 * in arrival order; whenever one of the server's slots is free, waiting
 * queries of the oldest request's index are gathered into one batch of at
 * most max_batch queries (across requests; a larger request is split over
 * several batches) and searched on that slot's stream, so batches of
 * different slots overlap on the device.  Each slot holds its own workspace
 * and buffers; the number of slots is `slots`, reduced to what mem_budget
 * bytes hold when mem_budget > 0 (OSANN_ERR_OOM when it holds none).  With
 * use_graphs, a batch is a CUDA graph replay (one graph per slot, index and
 * batch-size bucket 64, 128, ... max_batch, captured on first use, the batch
 * padded to its bucket with zero queries whose results are dropped).
 * Every query's result equals that of osann_search with the index's P and
 * k, bit for bit, whatever batch it ran in. */
typedef struct osann_server osann_server;

/* indexes[n_indexes] must outlive the server; P[i], k[i] (1..32) are index
 * i's probe budget and neighbour count. */
int osann_server_create(const osann_index *const *indexes, int32_t n_indexes, const int32_t *P, const int32_t *k,
                        int32_t slots, int64_t max_batch, size_t mem_budget, int32_t use_graphs,
                        osann_server **out);
/* Number of slots the memory budget allowed. */
int osann_server_slots(const osann_server *server);
/* Queue Q queries (device, Q x d of index `index`, ready on the device when
 * submitted, left untouched until the request finishes) whose results go to
 * the caller's device buffers d_ids (Q x k int64) and d_sqdists (Q x k fp32),
 * complete when the ticket is reported by osann_server_progress.
 * Non-blocking. */
int osann_server_submit(osann_server *server, int32_t index, const float *d_queries, int64_t Q, int64_t *d_ids,
                        float *d_sqdists, uint64_t *ticket);
/* Retire completed batches, admit waiting queries into free slots and
 * launch them; write up to max_done finished tickets to done and their
 * count to *n_done.  wait != 0 blocks on the oldest batch in flight when
 * nothing has finished yet. */
int osann_server_progress(osann_server *server, int32_t wait, uint64_t *done, int32_t max_done, int32_t *n_done);
/* Queries still waiting for a slot, and slots busy. */
int osann_server_pending(const osann_server *server, int64_t *waiting_queries, int32_t *busy_slots);
/* Autotuner: for every index and batch bucket, time each candidate (path,
 * work-list group size, screen layout) -- plain; batched with the default
 * and 32-query groups; fp16 screening with 128- and 64-query groups, and for
 * an index with 64 < d <= 128 with 128-query groups in both query-tile
 * layouts (OSANN_LAYOUT_SMEM, OSANN_LAYOUT_TMEM) -- on max_batch rows sampled
 * from the index itself, reps timed runs each, and keep the fastest.
 * out_choices (nullable) receives (path, group) per (index, bucket);
 * osann_server_choices gives the layouts too.  Call with no request in the
 * server. */
int osann_server_tune(osann_server *server, int32_t reps, int32_t *out_choices);
/* As osann_server_tune, timing each index i on the caller's sample queries
 * d_queries[i] (n_queries[i] rows, device; a NULL entry: rows of the index),
 * which tunes for the query distribution actually served. */
int osann_server_tune_queries(osann_server *server, const float *const *d_queries, const int64_t *n_queries,
                              int32_t reps, int32_t *out_choices);
/* The choice of every (index, bucket), index-major, as (path, group,
 * layout) triples: up to max_out triples into out3 (OSANN_LAYOUT_DEFAULT and
 * group 0 before tuning).  Returns the number of triples, 0 for a null
 * server. */
int osann_server_choices(const osann_server *server, int32_t *out3, int32_t max_out);
/* Run every slot, index and batch bucket once (capturing the graphs when
 * they are on), so that no capture happens while serving.  Call after
 * osann_server_tune (tuning drops the graphs) with no request in flight. */
int osann_server_warmup(osann_server *server);
/* Batch buckets in use (returns their count; writes up to max_out). */
int osann_server_buckets(const osann_server *server, int64_t *out, int32_t max_out);
/* Counters since creation: batches run, queries run (padding excluded),
 * graph replays, graphs captured, captures that failed (those batches run
 * directly). */
int osann_server_stats(const osann_server *server, int64_t out5[5]);
/* Synchronise the slots and release everything (NULL ok). */
int osann_server_free(osann_server *server);

#ifdef __cplusplus
}
#endif

#endif /* OSANN_H */
