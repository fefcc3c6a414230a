// libosann host library: the C ABI declared in include/osann.h.
//
// Validation, device allocation (stream-ordered, through an optional
// caller-installed allocator), per-device constant tables, workspace layout,
// the index build and the two search schedules, and stage timing.  Every
// step of the method runs in the kernels of keys.cu, buckets.cu, probes.cu,
// scan_plain.cu and scan_batched.cu; this file only sequences them.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "osann.h"
#include "osann_device.cuh"
#include "osann_launch.h"

// Binomial coefficients C(n, k), n <= MAX_D, k <= MAX_L, saturated at
// UINT64_MAX; used by the key (profile rank) and probe (unranking) kernels.
__device__ uint64_t g_binom_table[(osann::MAX_D + 1) * (osann::MAX_L + 1)];
// The same coefficients exact in 128 bits (low, high words): the ranks of
// the second-level table's 128-bit cone ids.
__device__ ulonglong2 g_binom_wide_table[(osann::MAX_D + 1) * (osann::MAX_L + 1)];
// Status word for the stateless entry points (osann_keys, osann_query_order).
__device__ uint32_t g_scratch_status[4];

namespace osann {

static thread_local char g_err[1024];
static std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// A thread capturing a search into a CUDA graph records no stage events;
// the kernels counted while capturing are credited per replay instead.
static thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

int count_launch()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OSANN_ERR_CUDA;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return 0;
}

static int cuda_fail(cudaError_t e, const char* what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return OSANN_ERR_CUDA;
}

// ---------------------------------------------------------------- allocator

static osann_alloc_fn g_alloc = nullptr;
static osann_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

// A block goes back to the allocator that gave it, even when the caller
// installs another allocator in between (an index built under one and
// freed under another): blocks of a caller's allocator are recorded with
// its release function.
struct CallerBlock {
    osann_free_fn fn;
    void* ctx;
};
static std::mutex g_blocks_mu;
static std::unordered_map<void*, CallerBlock> g_caller_blocks;

static void* dev_alloc(size_t bytes, cudaStream_t st)
{
    if (bytes == 0) bytes = 256;
    if (g_alloc) {
        void* p = g_alloc(bytes, st, g_alloc_ctx);
        if (p) {
            std::lock_guard<std::mutex> lk(g_blocks_mu);
            g_caller_blocks[p] = CallerBlock{g_free, g_alloc_ctx};
        }
        return p;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free(void* p, size_t bytes, cudaStream_t st)
{
    if (!p) return;
    CallerBlock b{nullptr, nullptr};
    bool caller = false;
    {
        std::lock_guard<std::mutex> lk(g_blocks_mu);
        auto it = g_caller_blocks.find(p);
        if (it != g_caller_blocks.end()) {
            b = it->second;
            caller = true;
            g_caller_blocks.erase(it);
        }
    }
    if (caller) {
        if (b.fn) b.fn(p, bytes, st, b.ctx);  // an allocator installed without a release function keeps its blocks
    } else {
        cudaFreeAsync(p, st);
    }
}

// ---------------------------------------------------------------- per device

struct DeviceState {
    bool ready = false;
    int num_sms = 0;
    uint64_t* binom = nullptr;
    ulonglong2* binom_w = nullptr;
    uint32_t* scratch_status = nullptr;
};
static DeviceState g_dev[64];
static std::mutex g_dev_mu;

static int device_state(DeviceState** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return OSANN_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceState& s = g_dev[dev];
    if (!s.ready) {
        std::vector<uint64_t> t((MAX_D + 1) * (MAX_L + 1), 0);
        for (int n = 0; n <= MAX_D; ++n)
            for (int k = 0; k <= MAX_L; ++k) {
                uint64_t v;
                if (k == 0) v = 1;
                else if (n == 0) v = 0;
                else {
                    uint64_t a = t[(n - 1) * (MAX_L + 1) + k - 1], b = t[(n - 1) * (MAX_L + 1) + k];
                    v = (a > UINT64_MAX - b) ? UINT64_MAX : a + b;
                }
                t[n * (MAX_L + 1) + k] = v;
            }
        if ((e = cudaMemcpyToSymbol(g_binom_table, t.data(), t.size() * sizeof(uint64_t))) != cudaSuccess)
            return cuda_fail(e, "binomial table upload");
        {
            // Pascal's rule in 128 bits: C(256, 16) < 2^84, so nothing saturates
            std::vector<unsigned __int128> w((MAX_D + 1) * (MAX_L + 1), 0);
            std::vector<ulonglong2> wt(w.size());
            for (int n = 0; n <= MAX_D; ++n)
                for (int k = 0; k <= MAX_L; ++k) {
                    unsigned __int128 v = k == 0 ? 1 : (n == 0 ? 0 : w[(n - 1) * (MAX_L + 1) + k - 1] +
                                                                        w[(n - 1) * (MAX_L + 1) + k]);
                    w[n * (MAX_L + 1) + k] = v;
                    wt[n * (MAX_L + 1) + k] = make_ulonglong2(uint64_t(v), uint64_t(v >> 64));
                }
            if ((e = cudaMemcpyToSymbol(g_binom_wide_table, wt.data(), wt.size() * sizeof(ulonglong2))) != cudaSuccess)
                return cuda_fail(e, "binomial table upload");
            if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.binom_w), g_binom_wide_table)) != cudaSuccess)
                return cuda_fail(e, "binomial table address");
        }
        if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.binom), g_binom_table)) != cudaSuccess)
            return cuda_fail(e, "binomial table address");
        if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scratch_status), g_scratch_status)) != cudaSuccess)
            return cuda_fail(e, "status word address");
        if ((e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "SM count");
        // keep stream-ordered allocations cached in this process's pool
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        s.ready = true;
    }
    *out = &s;
    return 0;
}

// ---------------------------------------------------------------- stats

struct StageRec {
    int stage;
    cudaEvent_t a, b;
};
static std::mutex g_stats_mu;
static bool g_stats_on = false;
static std::vector<StageRec> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
static double g_stage_ms[OSANN_NUM_STAGES];
static int64_t g_stage_n[OSANN_NUM_STAGES];

static cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct StageScope {
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageScope(int s, cudaStream_t stream) : stage(s), st(stream)
    {
        if (!g_stats_on || t_capturing) return;
        std::lock_guard<std::mutex> lk(g_stats_mu);
        a = take_event();
        cudaEventRecord(a, st);
    }
    ~StageScope()
    {
        if (!a) return;
        std::lock_guard<std::mutex> lk(g_stats_mu);
        cudaEvent_t b = take_event();
        cudaEventRecord(b, st);
        g_pending.push_back({stage, a, b});
    }
};

static void stats_collect()
{
    for (auto& r : g_pending) {
        float ms = 0.0f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        g_stage_ms[r.stage] += ms;
        g_stage_n[r.stage] += 1;
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_pending.clear();
}

}  // namespace osann

using namespace osann;

struct osann_index {
    // NC: cones of the CSR table (N_C for a direct table; min(N, N_C) + 1
    // compact cones for the second-level table); nc_clamp: N_C itself,
    // clamped to 2^62 (it bounds the probe budget)
    int64_t N = 0, NC = 0, max_bucket = 0, nc_clamp = 0;
    // occupied cones as counted by a synchronous build (0: unknown, e.g. an
    // asynchronous build); kept for the index's life, so the automatic path
    // choice -- and with it the workspace size -- never changes
    int64_t occupied = 0;
    unsigned __int128 nc_true = 0;
    bool hashed = false;          // second-level table (128-bit cone ids)
    int key_bits = 0;             // significant bits of the 128-bit ids
    uint4* ukeys = nullptr;       // [NC] 128-bit id of each compact cone (occupied ones first)
    uint32_t* htab = nullptr;     // open-addressing table: id -> compact cone
    uint32_t hmask = 0;
    const ulonglong2* binom_w = nullptr;
    // ROSANNA+: K centroids (K x d_pad, zero padded); cone ids are
    // cluster * ncc + cone of the residual (ncc = N_C of one cluster), and
    // nc_clamp bounds the budget per cluster
    int K = 0;
    float* cent = nullptr;
    unsigned __int128 ncc = 0;
    // temporaries kept by osann_rebuild after its first call (so that later
    // calls allocate nothing and can be captured in a CUDA graph)
    char* rb_temp = nullptr;
    size_t rb_temp_bytes = 0;
    float* rb_xr = nullptr;
    uint32_t* rb_asg = nullptr;
    int d = 0, d_pad = 0, L = 0, device = 0, num_sms = 0;
    int key_mode = OSANN_KEY_SET;  // OSANN_KEY_ORDERED: the members as a tuple in magnitude order
    cudaStream_t stream = nullptr;
    uint32_t* keys = nullptr;
    uint32_t* offsets = nullptr;
    uint32_t* perm = nullptr;
    float* xs = nullptr;
    float4* rowstat = nullptr;    // per row (1-B)|x|^2, |x|, |x|^2; N + TC_N rows
    // tensor-core screening operands per precision (0 bf16, 1 fp16): the
    // 16-bit scaled copy of xs, the extra K block of each row, the scale
    // (s, s^2, 1/s^2, X) and the TMA tensor maps over both arrays
    uint16_t* x16[2] = {nullptr, nullptr};
    uint16_t* xe16[2] = {nullptr, nullptr};
    float* tcs = nullptr;  // 2 x 4 floats
    bool tc_ready[2] = {false, false};
    alignas(64) unsigned char tmap[2][256];
    uint32_t* status = nullptr;   // [0] flags, [1] largest cone, [2] largest |x|^2 (bits)
    float* rot = nullptr;         // dk x d basis of the keys and query orders (null: the identity)
    float* rot_off = nullptr;     // dk offsets subtracted from the projected coordinates (null: none)
    int dk = 0;                   // key coordinates: d, or m for a projection
    unsigned long long* diag = nullptr;  // screening counters (survivors, fallbacks, checks, violations)
    uint64_t* binom = nullptr;
    float cdot2[2] = {0.f, 0.f}, cabs[2] = {0.f, 0.f}, Bn = 0.f;  // screening error-bound coefficients
    std::mutex tc_mu;
    std::vector<std::pair<void*, size_t>> allocs;
};

namespace osann {
// The permuted fp32 rows of an index (the request server samples them as
// tuning queries).
const float* index_rows(const osann_index* ix, int64_t* N, int* d, int* d_pad)
{
    *N = ix->N;
    *d = ix->d;
    *d_pad = ix->d_pad;
    return ix->xs;
}
int index_device(const osann_index* ix) { return ix->device; }
}  // namespace osann

// Coefficients of the screening bound
//     E = cdot2 |q||x| + Bn (|q|^2 + |x|^2) + cabs (|q| + |x|):
// 16-bit rounding of both operands (unit roundoff u = 2^-8 for bf16, 2^-11
// for fp16) and the fp32 accumulation of d_pad products (taken as
// d_pad 2^-20, sixteen times the round-to-nearest bound); for Bn the fp32
// norms, the accumulation of the folded norm terms over d_pad + 16 columns,
// their 16-bit hi/lo split (2^-15) and a cushion of 4e-6 for the fp32
// rounding of the exact distances compared at the end; for cabs the
// absolute rounding error of fp16 subnormals (half spacing 2^-25, times
// 2 sqrt(d) from Cauchy-Schwarz, with a factor 4 to spare; bf16 has fp32's
// exponent range, so its term is negligible but kept nonzero).
static void screen_coefficients(int d_pad, int prec, float* cdot2, float* cabs, float* Bn)
{
    const double u = std::ldexp(1.0, prec == 0 ? -8 : -11);
    const double c = 2 * u + u * u + d_pad * std::ldexp(1.0, -20) * (1 + u) * (1 + u);
    *cdot2 = float(2 * c);
    *cabs = float(prec == 0 ? std::ldexp(1.0, -120) : std::ldexp(1.0, -22) * std::sqrt(double(d_pad)));
    *Bn = float(d_pad * std::ldexp(1.0, -23) + (d_pad + 16) * std::ldexp(1.0, -20) + std::ldexp(1.0, -15) + 4e-6);
}

// OSANN_DEBUG_CHECKS=1 makes the screening kernel verify its error bound
// against an fp32 dot product for one column per thread and tile.
static int debug_checks()
{
    const char* e = std::getenv("OSANN_DEBUG_CHECKS");
    return (e && e[0] && e[0] != '0') ? 1 : 0;
}

static void index_release(osann_index* ix)
{
    for (auto& a : ix->allocs) dev_free(a.first, a.second, ix->stream);
    ix->allocs.clear();
    delete ix;
}

template <class T>
static T* index_alloc(osann_index* ix, size_t count)
{
    const size_t bytes = count * sizeof(T);
    void* p = dev_alloc(bytes, ix->stream);
    if (p) ix->allocs.push_back({p, bytes});
    return static_cast<T*>(p);
}

// N_C = C(d, L) 2^L, exact in 128 bits (below 2^100 for d <= MAX_D, L <= MAX_L).
static int cone_count(int d, int L, unsigned __int128* nc)
{
    if (d < 1 || L < 1 || L > d) return OSANN_ERR_INVALID;
    if (L > MAX_L || d > MAX_D) return OSANN_ERR_INVALID;
    // C(d, L) by the multiplicative formula; every prefix quotient is exact
    unsigned __int128 c = 1;
    for (int i = 1; i <= L; ++i) c = c * (unsigned __int128)(d - L + i) / (unsigned __int128)i;
    *nc = c << L;
    return OSANN_OK;
}

// N_C when a direct table can hold it (N_C < 2^31), else an error code.
static int64_t cones_or_error(int d, int L)
{
    unsigned __int128 nc = 0;
    const int rc = cone_count(d, L, &nc);
    if (rc) return rc;
    if (nc >= ((unsigned __int128)1 << 31)) return OSANN_ERR_UNSUPPORTED;
    return int64_t(nc);
}

static int64_t p_eff(const osann_index* ix, int64_t P) { return P < ix->nc_clamp ? P : ix->nc_clamp; }
// clusters visited per query: M, at most K (1 without clusters)
static int clusters_of(const osann_index* ix, int32_t M) { return ix->K ? (M < ix->K ? M : ix->K) : 1; }

static int pad_dim(int d)
{
    if (d <= 16) return 16;
    int p = 32;
    while (p < d) p <<= 1;
    return p;
}

static inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int TC_N_ROWS = 128;  // rows per tensor-core tile (padding of rowstat)

// ---------------------------------------------------------------- workspace

struct WsLayout {
    size_t qorder, qsign, probes, partial, qcount, qoff, fill, nitems, item_off, qlist, items, counters, scan_temp;
    size_t yb, qstat, ubits, scnt, surv, ovf, hbuf, yrot, vcl, ptab;
    size_t qset;  // query sets of the tensor-core work list, or SIZE_MAX
    size_t total;
    int64_t max_items;
};

enum SearchMode { MODE_PLAIN = 0, MODE_BATCHED = 1, MODE_BF16 = 2, MODE_FP16 = 3 };

static bool tc_mode(int mode) { return mode == MODE_BF16 || mode == MODE_FP16; }

// Prepare the screening operands of a precision on first use (bf16; fp16 is
// made with the index).  Synchronises `st` once so that later searches on
// any stream see them.
static int ensure_tc(osann_index* ix, int prec, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(ix->tc_mu);
    if (ix->tc_ready[prec]) return 0;
    if (ix->d_pad > 128) {
        set_error("the tensor-core path needs d <= 128");
        return OSANN_ERR_UNSUPPORTED;
    }
    if (!ix->x16[prec]) {
        ix->x16[prec] = index_alloc<uint16_t>(ix, size_t(ix->N) * ix->d_pad);
        ix->xe16[prec] = index_alloc<uint16_t>(ix, size_t(ix->N) * 16);
        if (!ix->x16[prec] || !ix->xe16[prec]) {
            set_error("tensor-core operands: device allocation failed");
            return OSANN_ERR_OOM;
        }
    }
    int rc = launch_tc_rows(prec, ix->xs, ix->rowstat, ix->N, ix->d_pad, ix->status + 2, ix->tcs + 4 * prec,
                            ix->x16[prec], ix->xe16[prec], st, ix->num_sms);
    if (rc) return rc;
    if (tc_encode_rows_map(ix->tmap[prec], ix->x16[prec], ix->N, ix->d_pad, prec) != 0 ||
        tc_encode_rows_map(ix->tmap[prec] + tc_map_bytes() / 2, ix->xe16[prec], ix->N, 0, prec) != 0)
        return OSANN_ERR_UNSUPPORTED;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core operands");
    ix->tc_ready[prec] = true;
    return 0;
}

static int group_size(int d_pad) { return 128 / (d_pad == 16 ? 1 : d_pad / 32); }

// Side streams for independent stages of one search (fork on an event of the
// caller's stream, join back before the dependent stage): a small pool per
// device, chosen by the caller's stream, and a fork/join event pair per host
// thread.  Event fork/join is also how a capturing stream pulls the side
// stream into its CUDA graph.
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static int side_stream(int device, cudaStream_t caller, SideStream* out)
{
    constexpr int POOL = 8, MAXDEV = 64;
    static std::mutex mu;
    static cudaStream_t pool[MAXDEV][POOL] = {};
    thread_local int ev_dev[MAXDEV] = {};
    thread_local cudaEvent_t ev[MAXDEV][2] = {};
    if (device < 0 || device >= MAXDEV) return OSANN_ERR_UNSUPPORTED;
    const int slot = int((reinterpret_cast<uintptr_t>(caller) >> 4) % POOL);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pool[device][slot] && cudaStreamCreateWithFlags(&pool[device][slot], cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "side stream");
    }
    if (!ev_dev[device]) {
        if (cudaEventCreateWithFlags(&ev[device][0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[device][1], cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "side stream events");
        ev_dev[device] = 1;
    }
    out->st = pool[device][slot];
    out->fork = ev[device][0];
    out->join = ev[device][1];
    return 0;
}

// Queries per work-list item: the default, or `group` when it is in range
// (1..128 for the tensor-core screen, whose MMA tile has 128 query rows;
// 1..group_size for the fp32 tile scan, whose thread layout fixes the most).
static int item_group(const osann_index* ix, int mode, int group)
{
    const int gmax = tc_mode(mode) ? TC_GROUP : group_size(ix->d_pad);
    return group >= 1 && group <= gmax ? group : gmax;
}

// P_eff: probe slots per query (Mv lists of P_eff / Mv positions with
// clusters); Mv: key rows per query (the residuals on its Mv clusters)
static WsLayout ws_layout(const osann_index* ix, int64_t Q, int64_t P_eff, int k, int mode, int group = 0, int Mv = 1)
{
    WsLayout w{};
    w.qset = SIZE_MAX;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    const int64_t Qv = Q * Mv;
    w.qorder = take(size_t(Qv) * ix->dk);
    if (ix->rot || ix->K) w.yrot = take(size_t(Qv) * ix->dk * 4);
    if (ix->K) w.vcl = take(size_t(Qv) * 4);
    w.qsign = take(size_t(Qv) * (MAX_D / 32) * 4);
    w.probes = take(size_t(Q) * P_eff * 4);
    w.ptab = take(probe_table_bytes(P_eff));
    if (mode != MODE_PLAIN) {
        const int G = item_group(ix, mode, group);
        const int64_t n = Q * P_eff;
        int64_t mi = n / G + ix->NC + 1;
        if (mi > n) mi = n;
        w.max_items = mi;
        if (mode == MODE_BATCHED) w.partial = take(size_t(n) * k * 8);
        w.qcount = take(size_t(ix->NC + 1) * 4);
        w.qoff = take(size_t(ix->NC + 1) * 4);
        w.fill = take(size_t(ix->NC + 1) * 4);
        w.nitems = take(size_t(ix->NC + 1) * 4);
        w.item_off = take(size_t(ix->NC + 1) * 4);
        w.qlist = take(size_t(n) * 4);
        w.items = take(size_t(mi > 0 ? mi : 1) * 16);
        w.counters = take(256);
        w.hbuf = take(size_t(wl_hist_entries(ix->NC, n, ix->num_sms)) * 4 + 4);
        const int64_t qw = tc_mode(mode) ? wl_qset_words(ix->NC, Q) : 0;
        w.qset = qw > 0 ? take(size_t(qw) * 4) : SIZE_MAX;
        w.scan_temp = take(batched_scan_temp_bytes(ix->NC, n, ix->num_sms));
    }
    if (tc_mode(mode)) {
        w.yb = take(size_t(Q) * ix->d_pad * 2);
        w.qstat = take(size_t(Q) * 16);
        w.ubits = take(size_t(Q) * 4);
        w.scnt = take(size_t(Q) * 4);
        w.surv = take(size_t(Q) * TC_SURV_CAP * 4);
        w.ovf = take(size_t(Q + 1) * 4);
    }
    w.total = off + 256;
    return w;
}

static int choose_mode(const osann_index* ix, int64_t Q, int64_t P_eff, int path)
{
    if (path == OSANN_PATH_PLAIN) return MODE_PLAIN;
    if (path == OSANN_PATH_BATCHED) return MODE_BATCHED;
    if (path == OSANN_PATH_BF16) return MODE_BF16;
    if (path == OSANN_PATH_FP16) return MODE_FP16;
    // queries per probed cone decide whether cone-major batching pays (over
    // the occupied cones when the build counted them: thin or skewed data
    // leaves most cones empty); the candidates per query decide whether one
    // CTA per query (plain) finishes soon enough: a small batch with a large
    // budget goes cone-major too.  The 16-bit screen beats the fp32 tile scan
    // wherever cone-major pays (measured on Gaussian and descriptor data,
    // thin cones included); the fp32 tile scan serves d_pad > 128
    const double cones = ix->occupied > 0 ? double(ix->occupied) : double(ix->NC);
    const double per_cone = double(Q) * double(P_eff) / cones;
    const double per_query = double(P_eff) * double(ix->N) / double(ix->NC);
    const bool big_queries = per_query >= 16384.0;
    if (ix->tc_ready[1] && (per_cone >= 8.0 || big_queries)) return MODE_FP16;
    return per_cone >= 16.0 || big_queries ? MODE_BATCHED : MODE_PLAIN;
}

// ---------------------------------------------------------------- C ABI

extern "C" {

int osann_set_allocator(osann_alloc_fn alloc, osann_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("allocator and free function must be set together");
        return OSANN_ERR_INVALID;
    }
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return OSANN_OK;
}

int osann_num_cones(int32_t d, int32_t L, int64_t* nc)
{
    int64_t r = cones_or_error(d, L);
    if (r < 0) {
        set_error("no cone count for d=%d L=%d", d, L);
        return int(r);
    }
    if (nc) *nc = r;
    return OSANN_OK;
}

const char* osann_last_error(void) { return g_err; }

int64_t osann_launch_count(void) { return g_launches.load(); }

int osann_debug_wait_budget(int64_t cycles)
{
    if (cycles < 0) {
        set_error("osann_debug_wait_budget: negative budget %lld", (long long)cycles);
        return OSANN_ERR_INVALID;
    }
    set_plain_wait_budget(cycles);
    return OSANN_OK;
}

int osann_stats_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_stats_on = on != 0;
    return OSANN_OK;
}

int osann_stats_reset(void)
{
    std::lock_guard<std::mutex> lk(g_stats_mu);
    stats_collect();
    for (int i = 0; i < OSANN_NUM_STAGES; ++i) {
        g_stage_ms[i] = 0;
        g_stage_n[i] = 0;
    }
    return OSANN_OK;
}

int osann_stats_get(int32_t stage, double* total_ms, int64_t* count)
{
    if (stage < 0 || stage >= OSANN_NUM_STAGES) return OSANN_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_stats_mu);
    stats_collect();
    if (total_ms) *total_ms = g_stage_ms[stage];
    if (count) *count = g_stage_n[stage];
    return OSANN_OK;
}

int osann_keys(const float* d_vectors, int64_t n, int32_t d, int32_t L, uint32_t* d_keys, void* stream)
{
    int64_t nc = cones_or_error(d, L);
    if (nc < 0 || n < 0 || (n > 0 && (!d_vectors || !d_keys))) {
        set_error("osann_keys: invalid arguments");
        return nc < 0 ? int(nc) : OSANN_ERR_INVALID;
    }
    DeviceState* ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    return launch_data_keys(d_vectors, n, d, L, ds->binom, d_keys, ds->scratch_status, nullptr,
                            static_cast<cudaStream_t>(stream), ds->num_sms);
}

int osann_keys_wide(const float* d_vectors, int64_t n, int32_t d, int32_t L, uint32_t* d_ids, void* stream)
{
    unsigned __int128 nc = 0;
    if (cone_count(d, L, &nc) != OSANN_OK || n < 0 || (n > 0 && (!d_vectors || !d_ids))) {
        set_error("osann_keys_wide: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    if (reinterpret_cast<uintptr_t>(d_ids) & 15) {
        set_error("osann_keys_wide: output must be 16-byte aligned");
        return OSANN_ERR_INVALID;
    }
    DeviceState* ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    return launch_data_keys(d_vectors, n, d, L, ds->binom, nullptr, ds->scratch_status, nullptr,
                            static_cast<cudaStream_t>(stream), ds->num_sms, ds->binom_w,
                            reinterpret_cast<uint4*>(d_ids));
}

int osann_query_order(const float* d_queries, int64_t Q, int32_t d, uint8_t* d_order, uint32_t* d_signs, void* stream)
{
    if (d < 1 || d > MAX_D || Q < 0 || (Q > 0 && (!d_queries || !d_order || !d_signs))) {
        set_error("osann_query_order: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    DeviceState* ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    return launch_query_order(d_queries, Q, d, d_order, d_signs, ds->scratch_status,
                              static_cast<cudaStream_t>(stream));
}

// Temporaries of one build: direct table (counts, scan, radix) or
// second-level table (128-bit ids, wide radix sort, run heads and their
// scan); plus the key-basis rows (a basis or centroids) and the points'
// clusters.
struct BuildTemps {
    size_t counts_bytes = 0, scan_bytes = 0, radix_bytes = 0, table_bytes = 0, total = 0;
    size_t xr_bytes = 0, asg_bytes = 0;
};
static BuildTemps build_temps(const osann_index* ix)
{
    BuildTemps t;
    const int64_t N = ix->N, NC = ix->NC;
    t.counts_bytes = ix->hashed ? 0 : al256(size_t(NC + 1) * 4);
    t.scan_bytes = ix->hashed ? al256(size_t(N) * 16) : al256(scan_temp_bytes(NC + 1));
    t.radix_bytes = ix->hashed ? al256(radix_temp_bytes_wide(N, ix->key_bits)) : al256(radix_temp_bytes(N, NC));
    t.table_bytes = ix->hashed ? al256(cone_table_temp_bytes(N)) : 0;
    t.total = t.counts_bytes + t.scan_bytes + t.radix_bytes + t.table_bytes;
    if (ix->rot || ix->K) t.xr_bytes = size_t(N) * ix->dk * 4;
    if (ix->K) t.asg_bytes = size_t(N) * 4;
    return t;
}

// Every kernel of a build, in stream order, into the index's buffers (the
// basis or centroids already in the index); temp, xr and asg as sized by
// build_temps.  Allocates nothing.
static int enqueue_build(osann_index* ix, const float* d_data, char* temp, float* xr, uint32_t* asg, cudaStream_t st)
{
    const BuildTemps t = build_temps(ix);
    const int64_t N = ix->N, NC = ix->NC;
    const int d = ix->d, m = ix->dk, L = ix->L, K = ix->K;
    const bool hashed = ix->hashed;
    const bool tc_possible = ix->d_pad <= 128;
    uint32_t* counts = reinterpret_cast<uint32_t*>(temp);
    void* scan_temp = temp + t.counts_bytes;
    void* radix_temp = temp + t.counts_bytes + t.scan_bytes;
    void* table_temp = temp + t.counts_bytes + t.scan_bytes + t.radix_bytes;
    uint4* wkeys = hashed ? static_cast<uint4*>(scan_temp) : nullptr;  // 128-bit ids of the rows
    int rc = 0;
    cudaMemsetAsync(ix->status, 0, 64 * 4, st);
    cudaMemsetAsync(ix->diag, 0, 8 * sizeof(unsigned long long), st);
    cudaMemsetAsync(ix->rowstat + N, 0, TC_N_ROWS * sizeof(float4), st);
    if (!hashed) cudaMemsetAsync(counts, 0, size_t(NC + 1) * 4, st);
    {
        StageScope s(OSANN_STAGE_DATA_KEYS, st);
        // keys come from the rows' coordinates on the index's basis
        const float* key_src = d_data;
        if (K > 0) {
            // ROSANNA+: each point's nearest centroid, then its residual
            rc = launch_nearest_centroids(d_data, N, d, ix->d_pad, ix->cent, K, 1, asg, st);
            if (!rc) rc = launch_residual_rows(d_data, N, d, ix->cent, ix->d_pad, asg, 1, xr, st, ix->num_sms);
            key_src = xr;
        } else if (ix->rot) {
            rc = launch_rotate_rows(ix->rot, ix->rot_off, d_data, N, d, m, xr, st, ix->num_sms);
            key_src = xr;
        }
        if (!rc)
            rc = launch_data_keys(key_src, N, m, L, ix->binom, ix->keys, ix->status, ix->status + 2, st, ix->num_sms,
                                  ix->binom_w, wkeys, ix->key_mode == OSANN_KEY_ORDERED);
        if (!rc && K > 0)
            rc = launch_composite_keys(asg, N, uint64_t(ix->ncc), uint64_t(ix->ncc >> 64), ix->keys, wkeys, st,
                                       ix->num_sms);
        // the fp16 scale and the norm bound need the original rows' norms, which
        // a projection, an offset or a residual does not keep
        if (!rc && ((ix->rot && (m < d || ix->rot_off)) || K > 0)) {
            cudaMemsetAsync(ix->status + 2, 0, 4, st);
            rc = launch_row_norm_max(d_data, N, d, ix->status + 2, st, ix->num_sms);
        }
        if (!rc && tc_possible) rc = launch_tc_scale(1, ix->status + 2, ix->tcs + 4, st);
    }
    if (!rc) {
        StageScope s(OSANN_STAGE_BUCKETS, st);
        if (hashed) {
            rc = launch_stable_sort_wide(wkeys, N, ix->key_bits, ix->perm, radix_temp, st);
            if (!rc)
                rc = launch_cone_table(wkeys, ix->perm, N, NC, ix->keys, ix->offsets, ix->ukeys, ix->status + 4,
                                       ix->htab, ix->hmask, table_temp, st, ix->num_sms);
        } else if (radix_single_pass(NC)) {
            rc = launch_stable_sort_ids(ix->keys, N, NC, ix->perm, ix->offsets, radix_temp, st);
        } else {
            rc = launch_key_histogram(ix->keys, N, NC, counts, st, ix->num_sms);
            if (!rc) rc = launch_exclusive_scan(counts, ix->offsets, NC + 1, scan_temp, st);
            if (!rc) rc = launch_stable_sort_ids(ix->keys, N, NC, ix->perm, nullptr, radix_temp, st);
        }
    }
    if (!rc) {
        StageScope s(OSANN_STAGE_GATHER, st);
        rc = launch_gather_rows(d_data, N, d, ix->d_pad, ix->perm, ix->xs, ix->rowstat, ix->Bn,
                                tc_possible ? ix->tcs + 4 : nullptr, ix->x16[1], ix->xe16[1], st, ix->num_sms);
    }
    if (!rc) rc = launch_max_bucket(ix->offsets, NC, ix->status + 1, st, ix->status + 3);
    return rc;
}

static int build_impl(const float* d_data, int64_t N, int32_t d, int32_t L, const float* d_rot, const float* d_off,
                      int32_t m, void* stream, bool async, int32_t cone_table, osann_index** out,
                      const float* d_cent = nullptr, int32_t K = 0, int32_t key_mode = OSANN_KEY_SET)
{
    if (!d_rot) m = d;
    if (d_rot && (m < 1 || m > d || d > 128)) {
        set_error("osann_build_proj: need 1 <= m <= d <= 128 (m=%d d=%d)", m, d);
        return OSANN_ERR_INVALID;
    }
    if (!out || !d_data || N < 1) {
        set_error("osann_build: invalid arguments (data=%p N=%lld out=%p)", (const void*)d_data, (long long)N,
                  (void*)out);
        return OSANN_ERR_INVALID;
    }
    *out = nullptr;
    if (cone_table < OSANN_CONES_AUTO || cone_table > OSANN_CONES_HASHED) {
        set_error("osann_build: unknown cone table kind %d", cone_table);
        return OSANN_ERR_INVALID;
    }
    unsigned __int128 nc_true = 0;
    if (cone_count(m, L, &nc_true) != OSANN_OK) {
        set_error("osann_build: unsupported (d=%d, L=%d): need 1<=d<=%d, 1<=L<=min(d,%d)", m, L, MAX_D, MAX_L);
        return OSANN_ERR_INVALID;
    }
    if (key_mode != OSANN_KEY_SET && key_mode != OSANN_KEY_ORDERED) {
        set_error("osann_build: unknown key mode %d", key_mode);
        return OSANN_ERR_INVALID;
    }
    if (key_mode == OSANN_KEY_ORDERED) {
        // d!/(d-L)! 2^L in a direct table only, and no clusters
        unsigned __int128 f = 1;
        for (int i = 0; i < L && f < ((unsigned __int128)1 << 31); ++i) f *= (unsigned __int128)(m - i);
        nc_true = f << L;
        if (nc_true >= ((unsigned __int128)1 << 31) || cone_table == OSANN_CONES_HASHED || K > 0) {
            set_error("osann_build: the ORDERED key needs N_C = d!/(d-L)! 2^L < 2^31, a direct table and no "
                      "clusters (d=%d L=%d)", m, L);
            return OSANN_ERR_UNSUPPORTED;
        }
    }
    const unsigned __int128 ncc = nc_true;  // cones of one cluster
    if (K < 0 || (K > 0 && (!d_cent || d_rot || d > 128 || K > (1 << 24)))) {
        set_error("osann_build: clusters need 1 <= K <= 2^24 centroids, d <= 128 and no key basis (K=%d d=%d)", K, d);
        return OSANN_ERR_INVALID;
    }
    if (K > 0) nc_true *= (unsigned __int128)K;  // composite ids cluster * N_C + cone
    if (N >= (int64_t(1) << 31)) {
        set_error("osann_build: N=%lld exceeds 2^31-1", (long long)N);
        return OSANN_ERR_UNSUPPORTED;
    }
    // a direct table up to N_C < 2^31; beyond, the second-level table over
    // the at most min(N, N_C) occupied cones (plus one empty cone)
    const bool fits = nc_true < ((unsigned __int128)1 << 31);
    if (cone_table == OSANN_CONES_DENSE && !fits) {
        set_error("osann_build: N_C >= 2^31 (d=%d, L=%d) needs the second-level cone table", m, L);
        return OSANN_ERR_UNSUPPORTED;
    }
    const bool hashed = cone_table == OSANN_CONES_HASHED || (cone_table == OSANN_CONES_AUTO && !fits);
    const int64_t NC = hashed ? (nc_true < (unsigned __int128)N ? int64_t(nc_true) : N) + 1 : int64_t(nc_true);
    if (hashed && NC > (int64_t(1) << 30)) {
        set_error("osann_build: a second-level table holds at most 2^30 cones (N=%lld)", (long long)N);
        return OSANN_ERR_UNSUPPORTED;
    }
    int key_bits = 1;
    while (key_bits < 127 && ((unsigned __int128)1 << key_bits) < nc_true) ++key_bits;
    uint32_t hcap = 1;
    while (int64_t(hcap) < 2 * NC) hcap <<= 1;
    DeviceState* ds;
    int rc = device_state(&ds);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    osann_index* ix = new osann_index();
    ix->N = N;
    ix->NC = NC;
    ix->nc_true = nc_true;
    ix->nc_clamp = ncc < ((unsigned __int128)1 << 62) ? int64_t(ncc) : (int64_t(1) << 62);
    ix->K = K;
    ix->ncc = ncc;
    ix->hashed = hashed;
    ix->key_bits = key_bits;
    ix->hmask = hcap - 1;
    ix->binom_w = ds->binom_w;
    ix->d = d;
    ix->dk = m;
    ix->d_pad = pad_dim(d);
    ix->L = L;
    ix->key_mode = key_mode;
    ix->stream = st;
    ix->num_sms = ds->num_sms;
    ix->binom = ds->binom;
    cudaGetDevice(&ix->device);

    ix->keys = index_alloc<uint32_t>(ix, size_t(N));
    ix->offsets = index_alloc<uint32_t>(ix, size_t(NC + 1));
    ix->perm = index_alloc<uint32_t>(ix, size_t(N));
    ix->xs = index_alloc<float>(ix, size_t(N) * ix->d_pad);
    ix->rowstat = index_alloc<float4>(ix, size_t(N) + TC_N_ROWS);
    ix->status = index_alloc<uint32_t>(ix, 64);
    ix->diag = index_alloc<unsigned long long>(ix, 8);
    ix->tcs = index_alloc<float>(ix, 8);
    for (int p = 0; p < 2; ++p) screen_coefficients(ix->d_pad, p, &ix->cdot2[p], &ix->cabs[p], &ix->Bn);
    const bool tc_possible = ix->d_pad <= 128;
    if (tc_possible) {
        // the default screening precision (fp16) is prepared with the index
        ix->x16[1] = index_alloc<uint16_t>(ix, size_t(N) * ix->d_pad);
        ix->xe16[1] = index_alloc<uint16_t>(ix, size_t(N) * 16);
    }
    if (hashed) {
        ix->ukeys = index_alloc<uint4>(ix, size_t(NC));
        ix->htab = index_alloc<uint32_t>(ix, size_t(hcap));
    }
    if (K > 0) ix->cent = index_alloc<float>(ix, size_t(K) * ix->d_pad);
    if (d_rot) {
        ix->rot = index_alloc<float>(ix, size_t(m) * d);
        if (d_off) ix->rot_off = index_alloc<float>(ix, size_t(m));
    }
    const BuildTemps bt = build_temps(ix);
    char* temp = static_cast<char*>(dev_alloc(bt.total, st));
    float* xr = bt.xr_bytes ? static_cast<float*>(dev_alloc(bt.xr_bytes, st)) : nullptr;
    uint32_t* asg = bt.asg_bytes ? static_cast<uint32_t*>(dev_alloc(bt.asg_bytes, st)) : nullptr;
    auto free_temps = [&]() {
        if (temp) dev_free(temp, bt.total, st);
        if (xr) dev_free(xr, bt.xr_bytes, st);
        if (asg) dev_free(asg, bt.asg_bytes, st);
    };
    if (!ix->keys || !ix->offsets || !ix->perm || !ix->xs || !ix->rowstat || !ix->status ||
        !ix->diag || !ix->tcs || (tc_possible && (!ix->x16[1] || !ix->xe16[1])) ||
        (hashed && (!ix->ukeys || !ix->htab)) || (K > 0 && !ix->cent) || (d_rot && !ix->rot) ||
        (d_off && !ix->rot_off) || !temp || (bt.xr_bytes && !xr) || (bt.asg_bytes && !asg)) {
        free_temps();
        index_release(ix);
        set_error("osann_build: device allocation failed");
        return OSANN_ERR_OOM;
    }
    // the key basis or the centroids: the index keeps its own copy
    cudaError_t e = cudaSuccess;
    if (K > 0) {
        e = cudaMemsetAsync(ix->cent, 0, size_t(K) * ix->d_pad * 4, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(ix->cent, size_t(ix->d_pad) * 4, d_cent, size_t(d) * 4, size_t(d) * 4, size_t(K),
                                  cudaMemcpyDeviceToDevice, st);
    } else if (d_rot) {
        e = cudaMemcpyAsync(ix->rot, d_rot, size_t(m) * d * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && d_off)
            e = cudaMemcpyAsync(ix->rot_off, d_off, size_t(m) * 4, cudaMemcpyDeviceToDevice, st);
    }
    rc = e != cudaSuccess ? cuda_fail(e, "osann_build: basis") : enqueue_build(ix, d_data, temp, xr, asg, st);
    free_temps();
    // the tensor maps need only addresses and sizes: encode them while the device works
    const bool maps_ok = !rc && tc_possible && tc_map_bytes() <= sizeof(ix->tmap[1]) &&
                         tc_encode_rows_map(ix->tmap[1], ix->x16[1], N, ix->d_pad, 1) == 0 &&
                         tc_encode_rows_map(ix->tmap[1] + tc_map_bytes() / 2, ix->xe16[1], N, 0, 1) == 0;
    if (!rc && async) {
        // status (non-finite data, timeouts) and the largest cone are read by
        // the next osann_status call
        ix->max_bucket = -1;
        ix->tc_ready[1] = maps_ok;
        *out = ix;
        return OSANN_OK;
    }
    uint32_t host_status[4] = {0, 0, 0, 0};  // flags, largest cone, largest |x|^2, occupied cones
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(host_status, ix->status, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "osann_build");
    }
    if (!rc && (host_status[0] & ST_TIMEOUT)) {
        set_error("osann_build: a device wait timed out");
        rc = OSANN_ERR_TIMEOUT;
    }
    if (!rc && (host_status[0] & ST_NONFINITE_DATA)) {
        set_error("osann_build: data contains NaN or Inf");
        rc = OSANN_ERR_NONFINITE;
    }
    if (rc) {
        index_release(ix);
        return rc;
    }
    cudaMemsetAsync(ix->status, 0, 4, st);
    ix->max_bucket = host_status[1];
    ix->occupied = host_status[3];
    ix->tc_ready[1] = maps_ok;
    *out = ix;
    return OSANN_OK;
}

int osann_build(const float* d_data, int64_t N, int32_t d, int32_t L, void* stream, osann_index** out)
{
    return build_impl(d_data, N, d, L, nullptr, nullptr, d, stream, false, OSANN_CONES_AUTO, out);
}

int osann_build_async(const float* d_data, int64_t N, int32_t d, int32_t L, void* stream, osann_index** out)
{
    return build_impl(d_data, N, d, L, nullptr, nullptr, d, stream, true, OSANN_CONES_AUTO, out);
}

int osann_build_ex(const float* d_data, int64_t N, int32_t d, int32_t L, const osann_build_opts* opts, void* stream,
                   osann_index** out)
{
    if (!opts) return osann_build(d_data, N, d, L, stream, out);
    if (!opts->d_basis && opts->d_offset) {
        set_error("osann_build_ex: an offset needs a basis");
        return OSANN_ERR_INVALID;
    }
    return build_impl(d_data, N, d, L, opts->d_basis, opts->d_offset, opts->d_basis ? opts->m : d, stream,
                      opts->async != 0, opts->cone_table, out, opts->d_centroids, opts->n_clusters, opts->key_mode);
}

int osann_build_rot(const float* d_data, int64_t N, int32_t d, int32_t L, const float* d_rot, int32_t async,
                    void* stream, osann_index** out)
{
    if (!d_rot) {
        set_error("osann_build_rot: null basis");
        return OSANN_ERR_INVALID;
    }
    return build_impl(d_data, N, d, L, d_rot, nullptr, d, stream, async != 0, OSANN_CONES_AUTO, out);
}

int osann_build_proj(const float* d_data, int64_t N, int32_t d, int32_t L, const float* d_proj, const float* d_off,
                     int32_t m, int32_t async, void* stream, osann_index** out)
{
    if (!d_proj) {
        set_error("osann_build_proj: null projection");
        return OSANN_ERR_INVALID;
    }
    return build_impl(d_data, N, d, L, d_proj, d_off, m, stream, async != 0, OSANN_CONES_AUTO, out);
}

int osann_rebuild(osann_index* ix, const float* d_data, void* stream)
{
    if (!ix || !d_data) {
        set_error("osann_rebuild: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ix->rb_temp) {
        // first call: the build's temporaries become the index's own
        const BuildTemps bt = build_temps(ix);
        auto keep = [&](size_t bytes) -> void* {
            void* p = dev_alloc(bytes, st);
            if (p) ix->allocs.push_back({p, bytes});
            return p;
        };
        ix->rb_temp = static_cast<char*>(keep(bt.total));
        if (bt.xr_bytes) ix->rb_xr = static_cast<float*>(keep(bt.xr_bytes));
        if (bt.asg_bytes) ix->rb_asg = static_cast<uint32_t*>(keep(bt.asg_bytes));
        if (!ix->rb_temp || (bt.xr_bytes && !ix->rb_xr) || (bt.asg_bytes && !ix->rb_asg)) {
            set_error("osann_rebuild: device allocation failed");
            return OSANN_ERR_OOM;
        }
        ix->rb_temp_bytes = bt.total;
    }
    int rc = enqueue_build(ix, d_data, ix->rb_temp, ix->rb_xr, ix->rb_asg, st);
    // bf16 operands made by an earlier bf16 search follow the new rows
    if (!rc && ix->tc_ready[0])
        rc = launch_tc_rows(0, ix->xs, ix->rowstat, ix->N, ix->d_pad, ix->status + 2, ix->tcs, ix->x16[0],
                            ix->xe16[0], st, ix->num_sms);
    ix->max_bucket = -1;
    return rc;
}

int osann_free(osann_index* index)
{
    if (!index) return OSANN_OK;
    index_release(index);
    return OSANN_OK;
}

int osann_info(const osann_index* ix, int64_t* N, int32_t* d, int32_t* L, int64_t* NC, int64_t* max_bucket)
{
    if (!ix) {
        set_error("osann_info: null index");
        return OSANN_ERR_INVALID;
    }
    if (N) *N = ix->N;
    if (d) *d = ix->d;
    if (L) *L = ix->L;
    if (NC) *NC = ix->NC;
    if (max_bucket) *max_bucket = ix->max_bucket;
    return OSANN_OK;
}

int osann_export(const osann_index* ix, uint32_t* d_keys, uint32_t* d_offsets, uint32_t* d_perm, void* stream)
{
    if (!ix) {
        set_error("osann_export: null index");
        return OSANN_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (d_keys && e == cudaSuccess)
        e = cudaMemcpyAsync(d_keys, ix->keys, size_t(ix->N) * 4, cudaMemcpyDeviceToDevice, st);
    if (d_offsets && e == cudaSuccess)
        e = cudaMemcpyAsync(d_offsets, ix->offsets, size_t(ix->NC + 1) * 4, cudaMemcpyDeviceToDevice, st);
    if (d_perm && e == cudaSuccess)
        e = cudaMemcpyAsync(d_perm, ix->perm, size_t(ix->N) * 4, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? OSANN_OK : cuda_fail(e, "osann_export");
}

int osann_cones(const osann_index* ix, int32_t* hashed, uint64_t* n_cones, int64_t* table_cones, int64_t* occupied,
                void* stream)
{
    if (!ix) {
        set_error("osann_cones: null index");
        return OSANN_ERR_INVALID;
    }
    if (hashed) *hashed = ix->hashed ? 1 : 0;
    if (n_cones) {
        n_cones[0] = uint64_t(ix->nc_true);
        n_cones[1] = uint64_t(ix->nc_true >> 64);
    }
    if (table_cones) *table_cones = ix->NC;
    if (occupied) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        uint32_t h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, ix->status + 3, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "osann_cones");
        *occupied = h;
    }
    return OSANN_OK;
}

int osann_export_cones(const osann_index* ix, uint32_t* d_ids, void* stream)
{
    if (!ix || !d_ids) {
        set_error("osann_export_cones: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    if (!ix->hashed) {
        set_error("osann_export_cones: the index has a direct cone table");
        return OSANN_ERR_INVALID;
    }
    cudaError_t e = cudaMemcpyAsync(d_ids, ix->ukeys, size_t(ix->NC) * 16, cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? OSANN_OK : cuda_fail(e, "osann_export_cones");
}

int osann_status(const osann_index* ix, void* stream, uint32_t* flags)
{
    if (!ix || !flags) {
        set_error("osann_status: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, ix->status, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ix->status, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "osann_status");
    *flags = h[0];
    // an index built asynchronously learns its largest cone here
    if (ix->max_bucket < 0) const_cast<osann_index*>(ix)->max_bucket = h[1];
    return OSANN_OK;
}

size_t osann_search_workspace_size_group(const osann_index* ix, int64_t Q, int32_t P, int32_t k, int32_t path,
                                         int32_t group)
{
    if (!ix || Q < 0 || P < 1 || k < 1 || k > MAX_K) return 0;
    if (path < 0 || path > OSANN_PATH_FP16 || group < 0) return 0;
    const int64_t P_eff = p_eff(ix, P);
    return ws_layout(ix, Q, P_eff, k, choose_mode(ix, Q, P_eff, path), group).total;
}

size_t osann_search_clusters_workspace_size(const osann_index* ix, int64_t Q, int32_t M, int32_t P, int32_t k,
                                            int32_t path)
{
    if (!ix || Q < 0 || M < 1 || P < 1 || k < 1 || k > MAX_K) return 0;
    if (path < 0 || path > OSANN_PATH_FP16) return 0;
    const int Mv = clusters_of(ix, M);
    const int64_t P_eff = Mv * p_eff(ix, P);
    return ws_layout(ix, Q, P_eff, k, choose_mode(ix, Q, P_eff, path), 0, Mv).total;
}

size_t osann_search_workspace_size(const osann_index* ix, int64_t Q, int32_t P, int32_t k, int32_t path)
{
    return osann_search_workspace_size_group(ix, Q, P, k, path, 0);
}

// Query keys and probe lists.  P_per: positions per key row; Mv: key rows
// per query (its Mv nearest clusters with ROSANNA+, else 1); the probe list
// of query q is rows q * Mv .. q * Mv + Mv - 1 in turn (Mv * P_per slots).
static int query_front(const osann_index* ix, const float* Y, int64_t Q, int64_t P_per, int Mv, const WsLayout& L,
                       char* w, bool init_partial, int k, cudaStream_t st)
{
    int rc = 0;
    const int64_t Qv = Q * Mv;
    uint32_t* vcl = ix->K ? reinterpret_cast<uint32_t*>(w + L.vcl) : nullptr;
    {
        StageScope s(OSANN_STAGE_QUERY_ORDER, st);
        // on a rotated basis the magnitude order is that of the query's coordinates there
        const float* Yk = Y;
        if (ix->rot) {
            rc = launch_rotate_rows(ix->rot, ix->rot_off, Y, Q, ix->d, ix->dk, reinterpret_cast<float*>(w + L.yrot), st,
                                    ix->num_sms);
            Yk = reinterpret_cast<const float*>(w + L.yrot);
        } else if (ix->K) {
            // ROSANNA+: the residuals on the query's Mv nearest clusters
            rc = launch_nearest_centroids(Y, Q, ix->d, ix->d_pad, ix->cent, ix->K, Mv, vcl, st);
            if (!rc)
                rc = launch_residual_rows(Y, Q, ix->d, ix->cent, ix->d_pad, vcl, Mv,
                                          reinterpret_cast<float*>(w + L.yrot), st, ix->num_sms);
            Yk = reinterpret_cast<const float*>(w + L.yrot);
        }
        if (!rc)
            rc = launch_query_order(Yk, Qv, ix->dk, reinterpret_cast<uint8_t*>(w + L.qorder),
                                    reinterpret_cast<uint32_t*>(w + L.qsign), ix->status, st);
    }
    if (rc) return rc;
    StageScope s(OSANN_STAGE_PROBES, st);
    ProbeMap pm{};
    pm.ordered = ix->key_mode == OSANN_KEY_ORDERED;
    if (ix->hashed) {
        pm.binom_w = ix->binom_w;
        pm.ukeys = ix->ukeys;
        pm.htab = ix->htab;
        pm.hmask = ix->hmask;
        pm.sentinel = uint32_t(ix->NC - 1);  // always empty
    }
    if (ix->K) {
        pm.M = Mv;
        pm.vcl = vcl;
        pm.ncc_lo = uint64_t(ix->ncc);
        pm.ncc_hi = uint64_t(ix->ncc >> 64);
    }
    return launch_probes(reinterpret_cast<uint8_t*>(w + L.qorder), reinterpret_cast<uint32_t*>(w + L.qsign), Qv, ix->dk,
                         ix->L, P_per, ix->binom, reinterpret_cast<uint32_t*>(w + L.ptab),
                         reinterpret_cast<uint32_t*>(w + L.probes),
                         init_partial ? reinterpret_cast<uint64_t*>(w + L.partial) : nullptr, k, st, pm);
}

int osann_probes(const osann_index* ix, const float* d_queries, int64_t Q, int32_t P, uint32_t* d_probes, void* d_ws,
                 size_t ws_bytes, void* stream)
{
    if (!ix || Q < 0 || P < 1 || (Q > 0 && (!d_queries || !d_probes))) {
        set_error("osann_probes: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    if (Q == 0) return OSANN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t P_eff = p_eff(ix, P);
    const WsLayout L = ws_layout(ix, Q, P_eff, 1, MODE_PLAIN);
    void* owned = nullptr;
    if (!d_ws) {
        owned = d_ws = dev_alloc(L.total, st);
        if (!d_ws) {
            set_error("osann_probes: workspace allocation failed");
            return OSANN_ERR_OOM;
        }
    } else if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) {
        set_error("osann_probes: workspace must be 256-byte aligned");
        return OSANN_ERR_INVALID;
    } else if (ws_bytes < L.total) {
        set_error("osann_probes: workspace too small (%zu < %zu)", ws_bytes, L.total);
        return OSANN_ERR_INVALID;
    }
    char* w = static_cast<char*>(d_ws);
    int rc = query_front(ix, d_queries, Q, P_eff, 1, L, w, false, 1, st);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(d_probes, w + L.probes, size_t(Q) * P_eff * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "osann_probes");
    }
    if (owned) dev_free(owned, L.total, st);
    return rc;
}

// overlap_from (nullable): an event recorded on `stream` before the index's
// build was enqueued; the query-side steps (magnitude orders, probe lists),
// which do not read the built index, then run on a side stream after that
// event only, beside the build, and join before the rest of the search.
static int search_impl(const osann_index* ix, const float* Y, const int64_t* src, int64_t Q, int32_t P, int32_t k,
                       int64_t grid_w, int32_t radius, int32_t path, void* d_ws, size_t ws_bytes, int64_t* ids,
                       float* dists, void* stream, int32_t group = 0, int32_t M = 1,
                       cudaEvent_t overlap_from = nullptr, int32_t layout = OSANN_LAYOUT_DEFAULT)
{
    if (!ix || Q < 0 || P < 1 || k < 1 || k > MAX_K || path < 0 || path > OSANN_PATH_FP16 || group < 0 || M < 1 ||
        layout < OSANN_LAYOUT_DEFAULT || layout > OSANN_LAYOUT_TMEM ||
        (Q > 0 && (!Y || !ids || !dists))) {
        set_error("osann_search: invalid arguments (Q=%lld P=%d k=%d path=%d)", (long long)Q, P, k, path);
        return OSANN_ERR_INVALID;
    }
    if (src && (grid_w < 1 || radius < 0)) {
        set_error("osann_search_excl: grid_w must be >= 1 and radius >= 0");
        return OSANN_ERR_INVALID;
    }
    if (ix->K && M > 32) {
        set_error("osann_search_clusters: at most 32 clusters per query (M=%d)", M);
        return OSANN_ERR_INVALID;
    }
    if (Q == 0) return OSANN_OK;
    const int Mv = clusters_of(ix, M);
    const int64_t P_per = p_eff(ix, P);
    const int64_t P_eff = Mv * P_per;  // probe slots per query
    if (Q * P_eff >= (int64_t(1) << 32)) {
        set_error("osann_search: Q * min(P, N_C) must stay below 2^32");
        return OSANN_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int mode = choose_mode(ix, Q, P_eff, path);
    const int prec = mode == MODE_FP16 ? 1 : 0;
    if (tc_mode(mode)) {
        int trc = ensure_tc(const_cast<osann_index*>(ix), prec, st);
        if (trc) return trc;
    }
    const bool batched = mode != MODE_PLAIN;
    const WsLayout L = ws_layout(ix, Q, P_eff, k, mode, group, Mv);
    // the query-side steps read neither the rows, nor a second-level table,
    // nor a basis or centroids of the index only with a plain direct table
    SideStream front{};
    if (overlap_from && !ix->hashed && !ix->rot && !ix->K) {
        int frc = side_stream(ix->device, st, &front);
        if (frc) return frc;
        if (cudaStreamWaitEvent(front.st, overlap_from, 0) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "osann_build_search: fork");
    }
    const cudaStream_t fst = front.st ? front.st : st;
    void* owned = nullptr;
    if (!d_ws) {
        owned = d_ws = dev_alloc(L.total, fst);  // usable on st after the join below
        if (!d_ws) {
            set_error("osann_search: workspace allocation failed (%zu bytes)", L.total);
            return OSANN_ERR_OOM;
        }
    } else if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) {
        set_error("osann_search: workspace must be 256-byte aligned");
        return OSANN_ERR_INVALID;
    } else if (ws_bytes < L.total) {
        set_error("osann_search: workspace too small (%zu < %zu)", ws_bytes, L.total);
        return OSANN_ERR_INVALID;
    }
    char* w = static_cast<char*>(d_ws);
    int rc = query_front(ix, Y, Q, P_per, Mv, L, w, mode == MODE_BATCHED, k, fst);
    if (front.st) {
        // join (also after an error, so that the side stream's work stays ordered before the caller's)
        if (cudaEventRecord(front.join, front.st) != cudaSuccess || cudaStreamWaitEvent(st, front.join, 0) != cudaSuccess)
            if (!rc) rc = cuda_fail(cudaGetLastError(), "osann_build_search: join");
    }
    if (!rc && batched) {
        BatchedBuffers b{};
        b.qcount = reinterpret_cast<uint32_t*>(w + L.qcount);
        b.qoff = reinterpret_cast<uint32_t*>(w + L.qoff);
        b.fill = reinterpret_cast<uint32_t*>(w + L.fill);
        b.nitems = reinterpret_cast<uint32_t*>(w + L.nitems);
        b.item_off = reinterpret_cast<uint32_t*>(w + L.item_off);
        b.qlist = reinterpret_cast<uint32_t*>(w + L.qlist);
        b.items = reinterpret_cast<uint4*>(w + L.items);
        b.hbuf = reinterpret_cast<uint32_t*>(w + L.hbuf);
        b.qset = L.qset != SIZE_MAX ? reinterpret_cast<uint32_t*>(w + L.qset) : nullptr;
        b.counters = reinterpret_cast<uint32_t*>(w + L.counters);
        b.n_items_dev = b.item_off + ix->NC;
        b.scan_temp = w + L.scan_temp;
        b.max_items = L.max_items;
        const int G = item_group(ix, mode, group);
        uint64_t* partial = reinterpret_cast<uint64_t*>(w + L.partial);
        const uint32_t* probes = reinterpret_cast<uint32_t*>(w + L.probes);
        // the query constants and seed bounds (tensor-core paths) and the work
        // list depend only on the probe lists: the former runs on a side stream
        SideStream side{};
        if (tc_mode(mode)) {
            rc = side_stream(ix->device, st, &side);
            if (!rc && (cudaEventRecord(side.fork, st) != cudaSuccess ||
                        cudaStreamWaitEvent(side.st, side.fork, 0) != cudaSuccess))
                rc = cuda_fail(cudaGetLastError(), "osann_search: fork");
            if (!rc) {
                StageScope s(OSANN_STAGE_TC_PREP, side.st);
                rc = launch_tc_query_prep(prec, Y, Q, ix->d, ix->d_pad, probes, P_eff, ix->offsets, uint32_t(ix->NC),
                                          ix->xs, k, ix->cdot2[prec], ix->cabs[prec], ix->tcs + 4 * prec, ix->perm,
                                          src, grid_w, radius, TC_SURV_CAP, w + L.yb,
                                          reinterpret_cast<float4*>(w + L.qstat),
                                          reinterpret_cast<uint32_t*>(w + L.ubits),
                                          reinterpret_cast<uint32_t*>(w + L.scnt), side.st);
            }
        }
        if (!rc) {
            StageScope s(OSANN_STAGE_WORKLIST, st);
            rc = launch_worklist(reinterpret_cast<uint32_t*>(w + L.probes), Q, P_eff, ix->offsets, ix->NC, G, b, st,
                                 ix->num_sms, tc_mode(mode));
        }
        if (side.st) {
            // join (also after an error, so that the side stream's work stays ordered before the caller's)
            if (cudaEventRecord(side.join, side.st) != cudaSuccess || cudaStreamWaitEvent(st, side.join, 0) != cudaSuccess)
                if (!rc) rc = cuda_fail(cudaGetLastError(), "osann_search: join");
        }
        if (!rc && tc_mode(mode)) {
            {
                StageScope s(OSANN_STAGE_TC_SCAN, st);
                rc = launch_tc_scan(prec, ix->tmap[prec], ix->perm, ix->rowstat, w + L.yb,
                                    reinterpret_cast<const float4*>(w + L.qstat), ix->tcs + 4 * prec, src, grid_w,
                                    radius, b, reinterpret_cast<uint32_t*>(w + L.ubits),
                                    reinterpret_cast<uint32_t*>(w + L.scnt), reinterpret_cast<uint32_t*>(w + L.surv),
                                    TC_SURV_CAP, ix->status, ix->diag, ix->xs, Y, P_eff, ix->d, ix->d_pad, k,
                                    ix->cdot2[prec], ix->Bn, ix->cabs[prec], debug_checks(), st, ix->num_sms,
                                    layout);
            }
            if (!rc) {
                StageScope s(OSANN_STAGE_TC_RERANK, st);
                rc = launch_tc_rerank(ix->xs, ix->d_pad, ix->perm, ix->offsets, uint32_t(ix->NC), Y, ix->d, Q, probes,
                                      P_eff, reinterpret_cast<uint32_t*>(w + L.scnt),
                                      reinterpret_cast<uint32_t*>(w + L.surv), TC_SURV_CAP, k, src, grid_w, radius,
                                      ix->diag, reinterpret_cast<uint32_t*>(w + L.ovf), ids, dists, st);
                // queries whose survivor list overflowed: exact scan of their probed cones
                if (!rc)
                    rc = launch_plain_scan(ix->xs, ix->offsets, ix->perm, ix->d_pad, Y, ix->d, Q, probes, P_eff,
                                           uint32_t(ix->NC), k, src, grid_w, radius,
                                           reinterpret_cast<const uint32_t*>(w + L.ovf), ix->num_sms, ids, dists,
                                           ix->status, st);
            }
        } else if (!rc) {
            {
                StageScope s(OSANN_STAGE_TILE_SCAN, st);
                rc = launch_tile_scan(ix->xs, ix->offsets, ix->perm, ix->d_pad, Y, ix->d, P_eff, k, src, grid_w,
                                      radius, b, G, partial, ix->status, st, ix->num_sms);
            }
            if (!rc) {
                StageScope s(OSANN_STAGE_MERGE, st);
                rc = launch_merge(partial, Q, P_eff, k, nullptr, ids, dists, st);
            }
        }
    } else if (!rc) {
        StageScope s(OSANN_STAGE_PLAIN_SCAN, st);
        rc = launch_plain_scan(ix->xs, ix->offsets, ix->perm, ix->d_pad, Y, ix->d, Q,
                               reinterpret_cast<uint32_t*>(w + L.probes), P_eff, uint32_t(ix->NC), k, src, grid_w,
                               radius, nullptr, ix->num_sms, ids, dists, ix->status, st);
    }
    if (owned) dev_free(owned, L.total, st);
    return rc;
}

int osann_search(const osann_index* index, const float* d_queries, int64_t Q, int32_t P, int32_t k, int32_t path,
                 void* d_ws, size_t ws_bytes, int64_t* d_ids, float* d_sqdists, void* stream)
{
    return search_impl(index, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream);
}

int osann_search_group(const osann_index* index, const float* d_queries, int64_t Q, int32_t P, int32_t k,
                       int32_t path, int32_t group, void* d_ws, size_t ws_bytes, int64_t* d_ids, float* d_sqdists,
                       void* stream)
{
    return search_impl(index, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream, group);
}

int osann_search_layout(const osann_index* index, const float* d_queries, int64_t Q, int32_t P, int32_t k,
                        int32_t path, int32_t group, int32_t layout, void* d_ws, size_t ws_bytes, int64_t* d_ids,
                        float* d_sqdists, void* stream)
{
    return search_impl(index, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream, group,
                       1, nullptr, layout);
}

int osann_search_clusters(const osann_index* index, const float* d_queries, int64_t Q, int32_t M, int32_t P,
                          int32_t k, int32_t path, void* d_ws, size_t ws_bytes, int64_t* d_ids, float* d_sqdists,
                          void* stream)
{
    return search_impl(index, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream, 0, M);
}

int osann_build_search(const float* d_data, int64_t N, int32_t d, int32_t L, const osann_build_opts* opts,
                       const float* d_queries, int64_t Q, int32_t P, int32_t k, int32_t path, void* d_ws,
                       size_t ws_bytes, int64_t* d_ids, float* d_sqdists, void* stream, osann_index** out)
{
    if (!out || !d_data || N < 1 || Q < 0 || (Q > 0 && (!d_queries || !d_ids || !d_sqdists))) {
        set_error("osann_build_search: invalid arguments");
        if (out) *out = nullptr;
        return OSANN_ERR_INVALID;
    }
    *out = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the fork point: everything enqueued before the build (the queries' producers)
    thread_local cudaEvent_t fork[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return OSANN_ERR_UNSUPPORTED;
    if (!fork[dev] && cudaEventCreateWithFlags(&fork[dev], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "osann_build_search: event");
    if (cudaEventRecord(fork[dev], st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "osann_build_search: fork");
    osann_build_opts o{};
    if (opts) o = *opts;
    const bool wait = o.async == 0;
    o.async = 1;  // the search is enqueued behind the build; its status is read at the end
    osann_index* ix = nullptr;
    int rc = osann_build_ex(d_data, N, d, L, &o, stream, &ix);
    if (rc) return rc;
    rc = search_impl(ix, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream, 0, 1,
                     fork[dev]);
    if (!rc && wait) {
        // the build's status, read without clearing (the search's own flags
        // stay for osann_status)
        uint32_t h[2] = {0, 0};
        cudaError_t e = cudaMemcpyAsync(h, ix->status, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "osann_build_search");
        } else {
            if (ix->max_bucket < 0) ix->max_bucket = h[1];
            if (h[0] & ST_TIMEOUT) {
                set_error("osann_build_search: a device wait timed out");
                rc = OSANN_ERR_TIMEOUT;
            } else if (h[0] & ST_NONFINITE_DATA) {
                set_error("osann_build_search: data contains NaN or Inf");
                rc = OSANN_ERR_NONFINITE;
            }
        }
    }
    if (rc) {
        if (!wait) cudaStreamSynchronize(st);  // nothing of the failed call may still use the index
        osann_free(ix);
        return rc;
    }
    *out = ix;
    return OSANN_OK;
}

int osann_rebuild_search(osann_index* ix, const float* d_data, const float* d_queries, int64_t Q, int32_t P,
                         int32_t k, int32_t path, void* d_ws, size_t ws_bytes, int64_t* d_ids, float* d_sqdists,
                         void* stream)
{
    if (!ix || !d_data || Q < 0 || (Q > 0 && (!d_queries || !d_ids || !d_sqdists))) {
        set_error("osann_rebuild_search: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    thread_local cudaEvent_t fork[64] = {};
    if (ix->device < 0 || ix->device >= 64) return OSANN_ERR_UNSUPPORTED;
    if (!fork[ix->device] && cudaEventCreateWithFlags(&fork[ix->device], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "osann_rebuild_search: event");
    // the fork point: everything enqueued before the rebuild (the queries' producers)
    if (cudaEventRecord(fork[ix->device], st) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "osann_rebuild_search: fork");
    int rc = osann_rebuild(ix, d_data, stream);
    if (rc) return rc;
    return search_impl(ix, d_queries, nullptr, Q, P, k, 0, 0, path, d_ws, ws_bytes, d_ids, d_sqdists, stream, 0, 1,
                       fork[ix->device]);
}

int osann_search_excl(const osann_index* index, const float* d_queries, const int64_t* d_query_src, int64_t Q,
                      int32_t P, int32_t k, int64_t grid_w, int32_t radius, int32_t path, void* d_ws, size_t ws_bytes,
                      int64_t* d_ids, float* d_sqdists, void* stream)
{
    if (!d_query_src && Q > 0) {
        set_error("osann_search_excl: null query source array");
        return OSANN_ERR_INVALID;
    }
    return search_impl(index, d_queries, d_query_src, Q, P, k, grid_w, radius, path, d_ws, ws_bytes, d_ids, d_sqdists,
                       stream);
}

int osann_screen_stats(const osann_index* ix, void* stream, int64_t* out4)
{
    if (!ix || !out4) {
        set_error("osann_screen_stats: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, ix->diag, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ix->diag, 0, sizeof(h), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "osann_screen_stats");
    for (int i = 0; i < 4; ++i) out4[i] = int64_t(h[i]);
    return OSANN_OK;
}

size_t osann_bruteforce_workspace_size(const osann_index* ix, int64_t Q, int32_t k)
{
    if (!ix || Q < 0 || k < 1 || k > MAX_K) return 0;
    return al256(bruteforce_ws_bytes(ix->N, ix->d_pad, Q, k)) + 256;
}

int osann_bruteforce(const osann_index* ix, const float* d_queries, const int64_t* d_query_src, int64_t Q, int32_t k,
                     int64_t grid_w, int32_t radius, void* d_ws, size_t ws_bytes, int64_t* d_ids, float* d_sqdists,
                     void* stream)
{
    if (!ix || Q < 0 || k < 1 || k > MAX_K || (Q > 0 && (!d_queries || !d_ids || !d_sqdists)) ||
        (d_query_src && (grid_w < 1 || radius < 0))) {
        set_error("osann_bruteforce: invalid arguments");
        return OSANN_ERR_INVALID;
    }
    if (Q == 0) return OSANN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t need = osann_bruteforce_workspace_size(ix, Q, k);
    void* owned = nullptr;
    if (!d_ws) {
        owned = d_ws = dev_alloc(need, st);
        if (!d_ws) {
            set_error("osann_bruteforce: workspace allocation failed");
            return OSANN_ERR_OOM;
        }
    } else if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) {
        set_error("osann_bruteforce: workspace must be 256-byte aligned");
        return OSANN_ERR_INVALID;
    } else if (ws_bytes < need) {
        set_error("osann_bruteforce: workspace too small (%zu < %zu)", ws_bytes, need);
        return OSANN_ERR_INVALID;
    }
    char* w = static_cast<char*>(d_ws);
    uint32_t* counter = reinterpret_cast<uint32_t*>(w + need - 256);
    int rc;
    {
        StageScope s(OSANN_STAGE_BRUTEFORCE, st);
        rc = launch_bruteforce_rows(ix->xs, ix->perm, ix->N, ix->d_pad, d_queries, ix->d, Q, k, d_query_src, grid_w,
                                    radius, w, counter, d_ids, d_sqdists, ix->status, st, ix->num_sms);
    }
    if (owned) dev_free(owned, need, st);
    return rc;
}

}  // extern "C"
