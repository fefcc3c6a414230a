// Continuous-batching request loop over indexes resident on the device.
//
// The paper has no counterpart: this is the serving layer around the search
// of Algorithm 1.  Requests (a block of queries for one index) wait in a
// FIFO; whenever one of the server's slots is free, the oldest waiting
// request's index is taken and as many waiting queries of that index as fit
// in one batch (max_batch) are gathered into the slot's query buffer, across
// requests and splitting large requests over several batches.  Each slot has
// its own stream, workspace and buffers, so batches of different slots
// overlap on the device; the number of slots is bounded by the memory budget
// (admission by memory).  A batch runs as a CUDA graph replay when graphs
// are on (one graph per slot, index and batch-size bucket, captured on first
// use; the batch is padded to the bucket with zero rows, whose results are
// discarded), and its path and work-list group size come
// from the tuner when it has run.  Results are copied to the callers'
// buffers on the slot's stream; a request is reported finished when the
// last of its batches has completed.  Every query's result is independent
// of the batch it ran in (all paths return the same bits), so a request's
// answer is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "osann.h"
#include "osann_launch.h"

namespace osann {
const float* index_rows(const osann_index* ix, int64_t* N, int* d, int* d_pad);
int index_device(const osann_index* ix);
}  // namespace osann

using namespace osann;

namespace {

constexpr int64_t MIN_BUCKET = 64;

struct Request {
    uint64_t ticket = 0;
    int index = 0;
    const float* q = nullptr;
    int64_t Q = 0, issued = 0, done = 0;
    int64_t* ids = nullptr;
    float* d2 = nullptr;
};

// queries [off, off + n) of request r, at rows [pos, pos + n) of the batch
struct Piece {
    Request* r;
    int64_t off, n, pos;
};

struct Choice {
    int path = OSANN_PATH_AUTO;
    int group = 0;
    int layout = OSANN_LAYOUT_DEFAULT;  // query tiles of the tensor-core screen
};

struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;  // kernels per replay
    bool failed = false;   // capture not possible: run directly
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    float* qbuf = nullptr;
    int64_t* ibuf = nullptr;
    float* dbuf = nullptr;
    bool busy = false;
    uint64_t seq = 0;
    std::vector<Piece> pieces;
    std::vector<Graph> graphs;  // [index * n_buckets + bucket]
};

}  // namespace

struct osann_server {
    std::vector<const osann_index*> idx;
    std::vector<int> P, k, d;
    int64_t max_batch = 0;
    int max_d = 0, max_k = 0, device = 0;
    std::vector<int64_t> buckets;
    std::vector<Choice> choice;  // [index * n_buckets + bucket]
    std::vector<Slot> slots;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> live;
    std::deque<uint64_t> finished;
    uint64_t next_ticket = 1, seq = 0;
    bool use_graphs = true;
    int64_t n_batches = 0, n_replays = 0, n_captured = 0, n_capture_failed = 0, n_queries = 0;
    std::mutex mu;
};

namespace {

int fail(int code, const char* msg)
{
    set_error("%s", msg);
    return code;
}

int cuda_err(cudaError_t e, const char* what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return OSANN_ERR_CUDA;
}

size_t nbuckets(const osann_server* s) { return s->buckets.size(); }

size_t bucket_of(const osann_server* s, int64_t n)
{
    size_t b = 0;
    while (b + 1 < s->buckets.size() && s->buckets[b] < n) ++b;
    return b;
}

// The candidate (path, group, layout) choices of the tuner; the workspace of
// a slot covers all of them.  The query-tile layout of the screen is a
// choice only where both exist (d_pad = 128: 64 < d <= 128).
std::vector<Choice> candidates(const osann_server* s, int i)
{
    int32_t d = 0;
    osann_info(s->idx[size_t(i)], nullptr, &d, nullptr, nullptr, nullptr);
    std::vector<Choice> c;
    c.push_back({OSANN_PATH_PLAIN, 0, OSANN_LAYOUT_DEFAULT});
    c.push_back({OSANN_PATH_BATCHED, 0, OSANN_LAYOUT_DEFAULT});
    c.push_back({OSANN_PATH_BATCHED, 32, OSANN_LAYOUT_DEFAULT});
    if (d > 64 && d <= 128) {
        c.push_back({OSANN_PATH_FP16, 128, OSANN_LAYOUT_TMEM});
        c.push_back({OSANN_PATH_FP16, 128, OSANN_LAYOUT_SMEM});
    } else {
        c.push_back({OSANN_PATH_FP16, 128, OSANN_LAYOUT_DEFAULT});
    }
    c.push_back({OSANN_PATH_FP16, 64, OSANN_LAYOUT_DEFAULT});
    return c;
}

int run_search(osann_server* s, Slot& sl, int i, int64_t n, const Choice& c)
{
    return osann_search_layout(s->idx[i], sl.qbuf, n, s->P[i], s->k[i], c.path, c.group, c.layout, sl.ws, sl.ws_bytes,
                               sl.ibuf, sl.dbuf, sl.st);
}

// One batch of `nq` queries of index i, already in the slot's query buffer.
int run_batch(osann_server* s, Slot& sl, int i, int64_t nq)
{
    const size_t b = bucket_of(s, nq);
    const Choice c = s->choice[size_t(i) * nbuckets(s) + b];
    if (!s->use_graphs) return run_search(s, sl, i, nq, c);
    Graph& g = sl.graphs[size_t(i) * nbuckets(s) + b];
    const int64_t nb = s->buckets[b];
    if (!g.exec && !g.failed) {
        set_capturing(true);
        const int64_t l0 = launch_total();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeRelaxed);
        int rc = e == cudaSuccess ? run_search(s, sl, i, nb, c) : OSANN_ERR_CUDA;
        if (e == cudaSuccess) {
            cudaError_t e2 = cudaStreamEndCapture(sl.st, &graph);
            if (e2 != cudaSuccess && rc == 0) rc = OSANN_ERR_CUDA;
        }
        set_capturing(false);
        const int64_t captured = launch_total() - l0;
        add_launches(-captured);
        if (rc == 0 && graph && cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess) {
            g.launches = captured;
            ++s->n_captured;
        } else {
            g.exec = nullptr;
            g.failed = true;
            ++s->n_capture_failed;
            cudaGetLastError();
        }
        if (graph) cudaGraphDestroy(graph);
    }
    if (g.failed) return run_search(s, sl, i, nq, c);
    // the padding rows are searched too (their results are dropped): zeros,
    // cheap and in range, rather than stale rows of another index or width
    if (nb > nq) {
        cudaError_t z = cudaMemsetAsync(sl.qbuf + nq * s->d[i], 0, size_t(nb - nq) * s->d[i] * 4, sl.st);
        if (z != cudaSuccess) return cuda_err(z, "osann_server: padding");
    }
    cudaError_t e = cudaGraphLaunch(g.exec, sl.st);
    if (e != cudaSuccess) return cuda_err(e, "osann_server: graph launch");
    add_launches(g.launches);
    ++s->n_replays;
    return 0;
}

void drop_graphs(osann_server* s)
{
    for (auto& sl : s->slots)
        for (auto& g : sl.graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = Graph{};
        }
}

// Retire the slots whose batch has completed.
int retire(osann_server* s)
{
    for (auto& sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) return cuda_err(e, "osann_server: batch");
        for (const Piece& p : sl.pieces) {
            p.r->done += p.n;
            if (p.r->done == p.r->Q) {
                s->finished.push_back(p.r->ticket);
                s->live.erase(p.r->ticket);
                delete p.r;
            }
        }
        sl.pieces.clear();
        sl.busy = false;
    }
    return 0;
}

// Fill free slots with batches of waiting queries.
int admit(osann_server* s)
{
    for (auto& sl : s->slots) {
        if (sl.busy) continue;
        if (s->pending.empty()) break;
        const int i = s->pending.front()->index;
        const int d = s->d[i], k = s->k[i];
        int64_t nq = 0;
        sl.pieces.clear();
        for (auto it = s->pending.begin(); it != s->pending.end() && nq < s->max_batch;) {
            Request* r = *it;
            if (r->index != i) {
                ++it;
                continue;
            }
            const int64_t take = std::min(r->Q - r->issued, s->max_batch - nq);
            sl.pieces.push_back({r, r->issued, take, nq});
            cudaError_t e = cudaMemcpyAsync(sl.qbuf + nq * d, r->q + r->issued * d, size_t(take) * d * 4,
                                            cudaMemcpyDeviceToDevice, sl.st);
            if (e != cudaSuccess) return cuda_err(e, "osann_server: query gather");
            r->issued += take;
            nq += take;
            if (r->issued == r->Q) it = s->pending.erase(it);
            else ++it;
        }
        int rc = run_batch(s, sl, i, nq);
        if (rc) return rc;
        ++s->n_batches;
        s->n_queries += nq;
        for (const Piece& p : sl.pieces) {
            cudaError_t e = cudaMemcpyAsync(p.r->ids + p.off * k, sl.ibuf + p.pos * k, size_t(p.n) * k * 8,
                                            cudaMemcpyDeviceToDevice, sl.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p.r->d2 + p.off * k, sl.dbuf + p.pos * k, size_t(p.n) * k * 4,
                                    cudaMemcpyDeviceToDevice, sl.st);
            if (e != cudaSuccess) return cuda_err(e, "osann_server: result scatter");
        }
        cudaError_t e = cudaEventRecord(sl.done, sl.st);
        if (e != cudaSuccess) return cuda_err(e, "osann_server: event");
        sl.busy = true;
        sl.seq = ++s->seq;
    }
    return 0;
}

void release(osann_server* s)
{
    drop_graphs(s);
    for (auto& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ws) cudaFree(sl.ws);
        if (sl.qbuf) cudaFree(sl.qbuf);
        if (sl.ibuf) cudaFree(sl.ibuf);
        if (sl.dbuf) cudaFree(sl.dbuf);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    for (Request* r : s->pending)
        if (s->live.count(r->ticket)) s->live.erase(r->ticket);
    for (auto& kv : s->live) delete kv.second;
    for (Request* r : s->pending) delete r;
    delete s;
}

}  // namespace

extern "C" {

int osann_server_create(const osann_index* const* indexes, int32_t n_indexes, const int32_t* P, const int32_t* k,
                        int32_t slots, int64_t max_batch, size_t mem_budget, int32_t use_graphs, osann_server** out)
{
    if (!out || !indexes || !P || !k || n_indexes < 1 || slots < 1 || max_batch < 1)
        return fail(OSANN_ERR_INVALID, "osann_server_create: invalid arguments");
    *out = nullptr;
    auto* s = new osann_server();
    s->max_batch = max_batch;
    s->use_graphs = use_graphs != 0;
    for (int i = 0; i < n_indexes; ++i) {
        int64_t N = 0;
        int d = 0, dp = 0;
        if (!indexes[i] || P[i] < 1 || k[i] < 1 || k[i] > 32) {
            delete s;
            return fail(OSANN_ERR_INVALID, "osann_server_create: bad index, P or k");
        }
        index_rows(indexes[i], &N, &d, &dp);
        if (i > 0 && index_device(indexes[i]) != index_device(indexes[0])) {
            delete s;
            return fail(OSANN_ERR_INVALID, "osann_server_create: indexes on different devices");
        }
        s->idx.push_back(indexes[i]);
        s->P.push_back(P[i]);
        s->k.push_back(k[i]);
        s->d.push_back(d);
        s->max_d = std::max(s->max_d, d);
        s->max_k = std::max(s->max_k, int(k[i]));
    }
    s->device = index_device(indexes[0]);
    for (int64_t b = MIN_BUCKET; b < max_batch; b *= 2) s->buckets.push_back(b);
    s->buckets.push_back(max_batch);
    s->choice.assign(size_t(n_indexes) * s->buckets.size(), Choice{});
    // one slot's memory: the largest workspace of any index, path and group the
    // server may run at the largest bucket, plus query and result buffers
    size_t ws = 0;
    for (int i = 0; i < n_indexes; ++i) {
        ws = std::max(ws, osann_search_workspace_size_group(s->idx[i], max_batch, P[i], k[i], OSANN_PATH_AUTO, 0));
        for (const Choice& c : candidates(s, i))
            ws = std::max(ws, osann_search_workspace_size_group(s->idx[i], max_batch, P[i], k[i], c.path, c.group));
    }
    const size_t qb = size_t(max_batch) * s->max_d * 4, ib = size_t(max_batch) * s->max_k * 8,
                 db = size_t(max_batch) * s->max_k * 4;
    const size_t per_slot = ws + qb + ib + db;
    int32_t n_slots = slots;
    if (mem_budget > 0) {
        const size_t fit = mem_budget / per_slot;
        if (fit < 1) {
            delete s;
            return fail(OSANN_ERR_OOM, "osann_server_create: the memory budget holds no slot");
        }
        if (fit < size_t(n_slots)) n_slots = int32_t(fit);
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    s->slots.resize(size_t(n_slots));
    cudaError_t e = cudaSuccess;
    for (auto& sl : s->slots) {
        sl.ws_bytes = ws;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.ws, ws);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.qbuf), qb);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.ibuf), ib);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.dbuf), db);
        // padded batch rows read the buffer's previous contents: start finite
        if (e == cudaSuccess) e = cudaMemsetAsync(sl.qbuf, 0, qb, sl.st);
        sl.graphs.assign(size_t(n_indexes) * s->buckets.size(), Graph{});
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaSetDevice(cur);
    if (e != cudaSuccess) {
        release(s);
        return e == cudaErrorMemoryAllocation ? fail(OSANN_ERR_OOM, "osann_server_create: device allocation failed")
                                              : cuda_err(e, "osann_server_create");
    }
    *out = s;
    return OSANN_OK;
}

int osann_server_slots(const osann_server* s) { return s ? int(s->slots.size()) : 0; }

int osann_server_submit(osann_server* s, int32_t index, const float* d_queries, int64_t Q, int64_t* d_ids,
                        float* d_sqdists, uint64_t* ticket)
{
    if (!s || !ticket || index < 0 || index >= int32_t(s->idx.size()) || Q < 0 ||
        (Q > 0 && (!d_queries || !d_ids || !d_sqdists)))
        return fail(OSANN_ERR_INVALID, "osann_server_submit: invalid arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    auto* r = new Request();
    r->ticket = s->next_ticket++;
    r->index = index;
    r->q = d_queries;
    r->Q = Q;
    r->ids = d_ids;
    r->d2 = d_sqdists;
    *ticket = r->ticket;
    if (Q == 0) {
        s->finished.push_back(r->ticket);
        delete r;
        return OSANN_OK;
    }
    s->live[r->ticket] = r;
    s->pending.push_back(r);
    return OSANN_OK;
}

int osann_server_progress(osann_server* s, int32_t wait, uint64_t* done, int32_t max_done, int32_t* n_done)
{
    if (!s || !n_done || max_done < 0 || (max_done > 0 && !done))
        return fail(OSANN_ERR_INVALID, "osann_server_progress: invalid arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    int rc = retire(s);
    if (!rc) rc = admit(s);
    if (!rc && wait && s->finished.empty()) {
        // block on the oldest batch in flight, then retire and refill
        Slot* oldest = nullptr;
        for (auto& sl : s->slots)
            if (sl.busy && (!oldest || sl.seq < oldest->seq)) oldest = &sl;
        if (oldest) {
            cudaError_t e = cudaEventSynchronize(oldest->done);
            if (e != cudaSuccess) rc = cuda_err(e, "osann_server: batch");
            if (!rc) rc = retire(s);
            if (!rc) rc = admit(s);
        }
    }
    cudaSetDevice(cur);
    int32_t n = 0;
    while (n < max_done && !s->finished.empty()) {
        done[n++] = s->finished.front();
        s->finished.pop_front();
    }
    *n_done = n;
    return rc;
}

int osann_server_pending(const osann_server* s, int64_t* waiting_queries, int32_t* busy_slots)
{
    if (!s) return fail(OSANN_ERR_INVALID, "osann_server_pending: null server");
    int64_t w = 0;
    for (const Request* r : s->pending) w += r->Q - r->issued;
    int32_t b = 0;
    for (const auto& sl : s->slots) b += sl.busy ? 1 : 0;
    if (waiting_queries) *waiting_queries = w;
    if (busy_slots) *busy_slots = b;
    return OSANN_OK;
}

int osann_server_tune_queries(osann_server* s, const float* const* d_queries, const int64_t* n_queries, int32_t reps,
                              int32_t* out_choices);

int osann_server_tune(osann_server* s, int32_t reps, int32_t* out_choices)
{
    return osann_server_tune_queries(s, nullptr, nullptr, reps, out_choices);
}

int osann_server_tune_queries(osann_server* s, const float* const* d_queries, const int64_t* n_queries, int32_t reps,
                              int32_t* out_choices)
{
    if (!s || reps < 1) return fail(OSANN_ERR_INVALID, "osann_server_tune: invalid arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    for (const auto& sl : s->slots)
        if (sl.busy) return fail(OSANN_ERR_INVALID, "osann_server_tune: batches in flight");
    if (!s->pending.empty()) return fail(OSANN_ERR_INVALID, "osann_server_tune: requests waiting");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    Slot& sl = s->slots[0];
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int rc = 0;
    const size_t nb = nbuckets(s);
    for (size_t i = 0; i < s->idx.size() && !rc; ++i) {
        // tuning queries: the caller's sample of index i, else max_batch rows
        // spread over the index (whose nearest neighbours are themselves: a
        // representative sample tunes better)
        int64_t N = 0;
        int d = 0, dp = 0;
        const float* rows = index_rows(s->idx[i], &N, &d, &dp);
        int64_t n = 0;
        if (d_queries && d_queries[i] && n_queries && n_queries[i] > 0) {
            n = std::min(s->max_batch, n_queries[i]);
            cudaError_t e = cudaMemcpyAsync(sl.qbuf, d_queries[i], size_t(n) * d * 4, cudaMemcpyDeviceToDevice, sl.st);
            if (e != cudaSuccess) rc = cuda_err(e, "osann_server_tune: sample");
        } else {
            n = std::min(s->max_batch, N);
            const int64_t step = n > 0 ? N / n : 1;
            if (n > 0) {
                cudaError_t e = cudaMemcpy2DAsync(sl.qbuf, size_t(d) * 4, rows, size_t(step) * dp * 4, size_t(d) * 4,
                                                  size_t(n), cudaMemcpyDeviceToDevice, sl.st);
                if (e != cudaSuccess) rc = cuda_err(e, "osann_server_tune: sample");
            }
        }
        for (size_t bk = 0; bk < nb && !rc; ++bk) {
            const int64_t q = std::min(s->buckets[bk], n);
            float best = -1.0f;
            Choice pick;
            for (const Choice& c : candidates(s, int(i))) {
                if (run_search(s, sl, int(i), q, c) != 0) {  // e.g. no fp16 operands for this index
                    cudaGetLastError();
                    continue;
                }
                float tot = 0.0f;
                bool ok = true;
                for (int r = 0; r < reps && ok; ++r) {
                    cudaEventRecord(a, sl.st);
                    ok = run_search(s, sl, int(i), q, c) == 0;
                    cudaEventRecord(b, sl.st);
                    float ms = 0.0f;
                    ok = ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
                    tot += ms;
                }
                if (ok && (best < 0.0f || tot < best)) {
                    best = tot;
                    pick = c;
                }
            }
            s->choice[i * nb + bk] = pick;
            if (out_choices) {
                out_choices[2 * (i * nb + bk)] = pick.path;
                out_choices[2 * (i * nb + bk) + 1] = pick.group;
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(sl.st);
    if (!rc && e != cudaSuccess) rc = cuda_err(e, "osann_server_tune");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    drop_graphs(s);  // captured with the previous choices
    cudaSetDevice(cur);
    return rc;
}

int osann_server_warmup(osann_server* s)
{
    if (!s) return fail(OSANN_ERR_INVALID, "osann_server_warmup: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    for (const auto& sl : s->slots)
        if (sl.busy) return fail(OSANN_ERR_INVALID, "osann_server_warmup: batches in flight");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    int rc = 0;
    // every slot, index and bucket once (captures the graphs when they are on);
    // the query buffers hold finite rows, whose results are dropped
    for (auto& sl : s->slots)
        for (size_t i = 0; i < s->idx.size() && !rc; ++i)
            for (size_t b = 0; b < s->buckets.size() && !rc; ++b) rc = run_batch(s, sl, int(i), s->buckets[b]);
    cudaError_t e = cudaDeviceSynchronize();
    if (!rc && e != cudaSuccess) rc = cuda_err(e, "osann_server_warmup");
    cudaSetDevice(cur);
    return rc;
}

int osann_server_choices(const osann_server* s, int32_t* out3, int32_t max_out)
{
    if (!s || (!out3 && max_out > 0)) return 0;
    const int32_t n = int32_t(s->choice.size());
    for (int32_t i = 0; i < n && i < max_out; ++i) {
        out3[3 * i] = s->choice[size_t(i)].path;
        out3[3 * i + 1] = s->choice[size_t(i)].group;
        out3[3 * i + 2] = s->choice[size_t(i)].layout;
    }
    return n;
}

int osann_server_buckets(const osann_server* s, int64_t* out, int32_t max_out)
{
    if (!s) return 0;
    const int32_t n = int32_t(s->buckets.size());
    for (int32_t i = 0; i < n && i < max_out; ++i) out[i] = s->buckets[i];
    return n;
}

int osann_server_stats(const osann_server* s, int64_t* out5)
{
    if (!s || !out5) return fail(OSANN_ERR_INVALID, "osann_server_stats: invalid arguments");
    out5[0] = s->n_batches;
    out5[1] = s->n_queries;
    out5[2] = s->n_replays;
    out5[3] = s->n_captured;
    out5[4] = s->n_capture_failed;
    return OSANN_OK;
}

int osann_server_free(osann_server* s)
{
    if (!s) return OSANN_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    release(s);
    cudaSetDevice(cur);
    return OSANN_OK;
}

}  // extern "C"
