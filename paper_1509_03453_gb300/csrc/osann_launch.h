// Host-side declarations of the kernel launchers (internal to libosann).
// Every launcher returns 0 or a negative OSANN_ERR_* code, and counts the
// kernels it launched.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace osann {

// Launch bookkeeping: checks cudaGetLastError, bumps the launch counter.
int count_launch();
void set_error(const char* fmt, ...);
// Graph capture: a capturing thread records no stage events; the launches
// counted while capturing are moved to the replays (add_launches).
void set_capturing(bool on);
void add_launches(int64_t n);
int64_t launch_total();

// keys.cu
// maxn2 may be null; wkeys non-null: 128-bit ids (four words per row) from
// the 128-bit binomial table binom_w instead of keys
// ordered: the ORDERED key (members as a tuple in magnitude order), direct table only
int launch_data_keys(const float* X, int64_t N, int d, int L, const uint64_t* binom, uint32_t* keys,
                     uint32_t* status, uint32_t* maxn2_bits, cudaStream_t st, int num_sms,
                     const ulonglong2* binom_w = nullptr, uint4* wkeys = nullptr, bool ordered = false);
// out (n x m) = rows of X on the m basis rows of Pm (m x d) minus off (null:
// none), fp32 in-order FMAs then one subtraction; d <= 128, m <= d (else -2)
int launch_rotate_rows(const float* Pm, const float* off, const float* X, int64_t n, int d, int m, float* out,
                       cudaStream_t st, int num_sms);
// atomicMax of the largest squared row norm into *maxn2_bits
int launch_row_norm_max(const float* X, int64_t n, int d, uint32_t* maxn2_bits, cudaStream_t st, int num_sms);
int launch_query_order(const float* Y, int64_t Q, int d, uint8_t* qorder, uint32_t* qsign, uint32_t* status,
                       cudaStream_t st);

// buckets.cu
size_t scan_temp_bytes(int64_t n);
int launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t st);
int launch_key_histogram(const uint32_t* keys, int64_t N, int64_t NC, uint32_t* counts, cudaStream_t st,
                         int num_sms);
size_t radix_temp_bytes(int64_t N, int64_t NC);
// offsets (nullable): with radix_single_pass(NC), also written: the CSR
// bucket starts (NC + 1 values), so no separate histogram is needed
bool radix_single_pass(int64_t NC);
int launch_stable_sort_ids(const uint32_t* keys, int64_t N, int64_t NC, uint32_t* perm, uint32_t* offsets, void* temp,
                           cudaStream_t st);
// LSD radix sort of the ids 0..N-1 by 128-bit key (key_bits significant
// bits), stable: perm[i] = the id at sorted position i
size_t radix_temp_bytes_wide(int64_t N, int key_bits);
int launch_stable_sort_wide(const uint4* wkeys, int64_t N, int key_bits, uint32_t* perm, void* temp, cudaStream_t st);
int launch_gather_rows(const float* X, int64_t N, int d, int d_pad, const uint32_t* perm, float* xs, float4* rowstat,
                       float Bn, const float* tcs, uint16_t* x16, uint16_t* xe16, cudaStream_t st,
                       int num_sms);  // tcs, x16, xe16 null: no fp16 operands
int launch_tc_scale(int prec, const uint32_t* maxn2_bits, float* tcs, cudaStream_t st);
// out_max: largest cone size (atomicMax); out_occ (nullable): occupied cones (atomicAdd)
int launch_max_bucket(const uint32_t* offsets, int64_t NC, uint32_t* out_max, cudaStream_t st,
                      uint32_t* out_occ = nullptr);

// cone_table.cu: the second-level table of occupied cones.  From perm
// (sorted by 128-bit id) and the ids: keys[row] = compact cone, offsets over
// the NCt compact cones (cones past the occupied ones are empty), ukeys[c] =
// the 128-bit id of compact cone c, the occupied count in *n_occ, and the
// hash table (hmask + 1 slots) from ids to compact cones.
size_t cone_table_temp_bytes(int64_t N);
int launch_cone_table(const uint4* wkeys, const uint32_t* perm, int64_t N, int64_t NCt, uint32_t* keys,
                      uint32_t* offsets, uint4* ukeys, uint32_t* n_occ, uint32_t* htab, uint32_t hmask, void* temp,
                      cudaStream_t st, int num_sms);

// probes.cu
// How probed cone ids become table cones.  Second-level table (htab non-null):
// 128-bit ids looked up, unoccupied ones to `sentinel`.  Clusters (vcl
// non-null, ROSANNA+): the Q rows of qorder/qsign are M residuals per query
// (row q * M + j on cluster vcl[q * M + j]), each with P_eff positions; the
// id is vcl * ncc + cone, and query q's list is its M lists in turn.
struct ProbeMap {
    bool ordered = false;  // the ORDERED key's profiles and ids (direct table only)
    const ulonglong2* binom_w = nullptr;
    const uint4* ukeys = nullptr;
    const uint32_t* htab = nullptr;
    uint32_t hmask = 0, sentinel = 0;
    int M = 1;
    const uint32_t* vcl = nullptr;
    uint64_t ncc_lo = 0, ncc_hi = 0;
};
// tab: scratch of probe_table_bytes(P_eff) for the per-position ranks and flips
size_t probe_table_bytes(int64_t P_eff);
int launch_probes(const uint8_t* qorder, const uint32_t* qsign, int64_t Q, int d, int L, int64_t P_eff,
                  const uint64_t* binom, uint32_t* tab, uint32_t* probes, uint64_t* partial, int k, cudaStream_t st,
                  const ProbeMap& pm = ProbeMap{});

// clusters.cu (ROSANNA+): nearest M of K centroids (K x d_pad, zero padded;
// d_pad <= 128, M <= min(K, 32)) by the canonical fp32 distance, ties to the
// lower index; residual rows X[v] - C[idx[v * M + j]]; composite ids
// asg * ncc + key (keys, or the 128-bit wkeys)
int launch_nearest_centroids(const float* X, int64_t n, int d, int d_pad, const float* C, int K, int M,
                             uint32_t* out, cudaStream_t st);
int launch_residual_rows(const float* X, int64_t n, int d, const float* C, int d_pad, const uint32_t* idx, int M,
                         float* out, cudaStream_t st, int num_sms);
int launch_composite_keys(const uint32_t* asg, int64_t N, uint64_t ncc_lo, uint64_t ncc_hi, uint32_t* keys,
                          uint4* wkeys, cudaStream_t st, int num_sms);

// scan_plain.cu
// clock budget of the plain scan's stage waits (0: the default, about a second)
void set_plain_wait_budget(long long cycles);
int launch_plain_scan(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad,
                      const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, uint32_t NC, int k,
                      const int64_t* query_src, int64_t grid_w, int radius, const uint32_t* qlist, int num_sms,
                      int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st);
// qlist (nullable): device list [count, q_0, ...] of the queries to scan

// scan_batched.cu
struct BatchedBuffers {
    uint32_t* qcount;     // NC + 1
    uint32_t* qoff;       // NC + 1
    uint32_t* fill;       // NC
    uint32_t* nitems;     // NC + 1
    uint32_t* item_off;   // NC + 1
    uint32_t* qlist;      // Q * P_eff
    uint4* items;         // max_items descriptors (first row, end row, first slot, slot count)
    uint32_t* hbuf;       // per-block cone histograms (N_C <= 12288)
    uint32_t* counters;   // word 0: work counter of the tile scan
    const uint32_t* n_items_dev;  // device word holding the item count (item_off + NC)
    void* scan_temp;
    int64_t max_items;
    uint32_t* qset;       // N_C x ceil(Q / 32) query-set words (query-only lists), or null
};
size_t batched_scan_temp_bytes(int64_t NC, int64_t n, int num_sms);
int wl_hist_entries(int64_t NC, int64_t n, int num_sms);
// Words of the query sets of a query-only work list (N_C <= 12288 and at
// most 256 MB), else 0.
int64_t wl_qset_words(int64_t NC, int64_t Q);
// probes: the query-major probe lists (slot q * P_eff + p = flat index);
// each cone's slots are grouped (ascending per chunk of the list).  Items are
// in cone order.  query_only (the tensor-core screen, which needs only each
// entry's query): with b.qset, the lists come from query sets, each cone's
// entries q * P_eff in ascending query order.
int launch_worklist(const uint32_t* probes, int64_t Q, int64_t P_eff, const uint32_t* offsets, int64_t NC,
                    int group, BatchedBuffers& b, cudaStream_t st, int num_sms, bool query_only = false);
int launch_tile_scan(const float* xs, const uint32_t* offsets, const uint32_t* perm, int d_pad, const float* Y,
                     int d, int64_t slots_per_query, int k, const int64_t* query_src, int64_t grid_w, int radius,
                     const BatchedBuffers& b, int group, uint64_t* partial, uint32_t* status, cudaStream_t st,
                     int num_sms);
int launch_merge(const uint64_t* partial, int64_t Q, int64_t slots, int k, const uint32_t* perm_or_null,
                 int64_t* out_ids, float* out_d, cudaStream_t st);

// linear search (scan_batched.cu): dense tile scan over all rows of xs
size_t bruteforce_ws_bytes(int64_t N, int d_pad, int64_t Q, int k);
int launch_bruteforce_rows(const float* xs, const uint32_t* perm, int64_t N, int d_pad, const float* Y, int d,
                           int64_t Q, int k, const int64_t* query_src, int64_t grid_w, int radius, void* ws,
                           uint32_t* counter, int64_t* out_ids, float* out_d, uint32_t* status, cudaStream_t st,
                           int num_sms);

// tc_scan.cu: 16-bit tensor-core screening + fp32 rerank.  prec 0 = bf16,
// 1 = fp16 (with an exact power-of-two scale of the data and queries)
constexpr int TC_GROUP = 128;
constexpr int TC_SURV_CAP = 1024;
size_t tc_map_bytes();
int tc_encode_rows_map(void* map_out, const void* x16, int64_t N, int d_pad, int prec);  // d_pad 0: extra block
int launch_tc_rows(int prec, const float* xs, const float4* rowstat, int64_t N, int d_pad, const uint32_t* maxn2_bits,
                   float* tcs, void* x16, void* xe16, cudaStream_t st, int num_sms);
int launch_tc_query_prep(int prec, const float* Y, int64_t Q, int d, int d_pad, const uint32_t* probes,
                         int64_t P_eff, const uint32_t* offsets, uint32_t NC, const float* xs, int k, float cdot2,
                         float cabs, const float* tcs, const uint32_t* perm, const int64_t* query_src, int64_t grid_w,
                         int radius, int cap, void* Y16, float4* qstat, uint32_t* Ubits, uint32_t* surv_cnt,
                         cudaStream_t st);
int launch_tc_scan(int prec, const void* maps, const uint32_t* perm, const float4* rowstat, const void* Y16,
                   const float4* qstat, const float* tcs, const int64_t* query_src, int64_t grid_w, int radius,
                   const BatchedBuffers& b, uint32_t* Ubits, uint32_t* surv_cnt, uint32_t* surv, int cap,
                   uint32_t* status, unsigned long long* diag, const float* xs, const float* Y, int64_t S, int d,
                   int d_pad, int k, float cdot2, float Bn, float cabs, int debug, cudaStream_t st, int num_sms,
                   int layout = 0);
int launch_tc_rerank(const float* xs, int d_pad, const uint32_t* perm, const uint32_t* offsets, uint32_t NC,
                     const float* Y, int d, int64_t Q, const uint32_t* probes, int64_t P_eff, const uint32_t* surv_cnt,
                     const uint32_t* surv, int cap, int k, const int64_t* query_src, int64_t grid_w, int radius,
                     unsigned long long* diag, uint32_t* ovf, int64_t* out_ids, float* out_d, cudaStream_t st);
// ovf: device list [count, q_0, ...] of the queries whose survivor list
// overflowed (Q + 1 words); they are left to the plain scan

}  // namespace osann
