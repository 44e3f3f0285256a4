// Serving engine: a request loop over one resident index.
//
// Requests (query batches and insertion batches, host buffers) are admitted
// in arrival order.  Every slot is a worker thread with its own CUDA stream,
// query context (search scratch) and pinned / device staging.  A free slot
// takes all consecutive queries at the head of the queue that fit its batch
// (continuous batching), so batches from several slots overlap on the GPU.
// An insertion is an epoch barrier: it is admitted only when it is at the
// head and no query batch is in flight, and queries behind it wait for it;
// hence every request observes exactly the insertions that arrived before it
// (labels are read by queries and written only by insertions).  Admission by
// memory: a slot's device scratch (its query context, sized for a full batch,
// and staging) is allocated when the slot is first needed, and only if the
// device's free memory at that moment (cudaMemGetInfo) leaves it within
// mem_fraction; until then the slot takes no work and requests wait for the
// slots that have memory.  The first slot is set up at creation.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "dbl_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int kind = 0;  // 0 query, 1 insertion
    const int32_t *a = nullptr, *b = nullptr;
    int64_t n = 0;
    uint8_t *ans = nullptr;
    Clock::time_point t_submit, t_done;
    dbl_status status = DBL_OK;
    bool done = false;
};

struct Slot {
    dbl_qctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int32_t *d_u = nullptr, *d_v = nullptr;
    uint8_t *d_ans = nullptr;
    int32_t *h_u = nullptr, *h_v = nullptr;
    uint8_t *h_ans = nullptr;
    bool ready = false;  // its scratch is allocated
    std::thread worker;
};

}  // namespace

struct dbl_server {
    dbl_index *ix = nullptr;
    int64_t max_batch = 0, max_pending = 0;
    int64_t per_slot = 0;       // device bytes one slot's scratch takes
    double mem_fraction = 0.5;  // share of the free device memory a new slot may take
    int64_t max_memory = 0;     // bytes all admitted slots may take together (0: no limit)
    int ready_slots = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::mutex setup_mu;        // one slot set-up at a time (each re-reads the free memory)
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    int queries_in_flight = 0;
    bool insert_in_flight = false;
    bool stop = false;
    uint64_t epoch = 0;
    std::vector<double> lat_q, lat_i;
    uint64_t queries_done = 0, edges_done = 0, batches = 0, batched_requests = 0, cancelled = 0;
    Clock::time_point t0;
    bool started = false;
    std::string err;
};

// A slot's scratch: stream, staging for max_batch pairs, and a query context
// sized for a full batch (so serving allocates nothing after this).
static dbl_status slot_setup(dbl_server *S, Slot &sl)
{
    dbl_index *ix = S->ix;
    const int64_t mb = S->max_batch;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) ||
        cudaMalloc(&sl.d_u, sizeof(int32_t) * mb) || cudaMalloc(&sl.d_v, sizeof(int32_t) * mb) ||
        cudaMalloc(&sl.d_ans, (size_t)mb) || cudaMallocHost(&sl.h_u, sizeof(int32_t) * mb) ||
        cudaMallocHost(&sl.h_v, sizeof(int32_t) * mb) || cudaMallocHost(&sl.h_ans, (size_t)mb)) {
        cudaGetLastError();
        return DBL_ERR_OOM;
    }
    dbl_status st = dbl_qctx_create(ix, &sl.ctx, sl.stream);
    if (!st) st = dbl::ensure_search_scratch(sl.ctx, mb, sl.stream);
    if (!st && cudaStreamSynchronize(sl.stream) != cudaSuccess) st = DBL_ERR_CUDA;
    if (!st) sl.ready = true;
    return st;
}

static void slot_release(Slot &sl)
{
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) dbl_qctx_destroy(sl.ctx, sl.stream);
    sl.ctx = nullptr;
    cudaFree(sl.d_u);
    cudaFree(sl.d_v);
    cudaFree(sl.d_ans);
    cudaFreeHost(sl.h_u);
    cudaFreeHost(sl.h_v);
    cudaFreeHost(sl.h_ans);
    sl.d_u = sl.d_v = nullptr;
    sl.d_ans = nullptr;
    sl.h_u = sl.h_v = nullptr;
    sl.h_ans = nullptr;
    if (sl.stream) cudaStreamDestroy(sl.stream);
    sl.stream = nullptr;
    sl.ready = false;
}

// Admission by memory: a slot without scratch sets it up when there is work
// and the device's free memory now leaves one more slot within mem_fraction.
// Returns false when the worker should stop.
static bool admit_slot(dbl_server *S, Slot *slot)
{
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || !S->pending.empty(); });
        if (S->stop && S->pending.empty()) return false;
        if (S->pending.empty()) return true;
    }
    std::lock_guard<std::mutex> g(S->setup_mu);
    size_t free_b = 0, total_b = 0;
    int ready = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ready = S->ready_slots;
    }
    const bool in_budget = S->max_memory <= 0 || (int64_t)(ready + 1) * S->per_slot <= S->max_memory;
    if (in_budget && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
        (double)S->per_slot <= S->mem_fraction * (double)free_b) {
        if (slot_setup(S, *slot) == DBL_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            ++S->ready_slots;
        } else {
            slot_release(*slot);
        }
    }
    if (!slot->ready) std::this_thread::sleep_for(std::chrono::microseconds(500));  // the other slots serve
    S->cv_work.notify_all();
    return true;
}

static void serve_worker(dbl_server *S, Slot *slot)
{
    dbl_index *ix = S->ix;
    for (;;) {
        if (!slot->ready) {
            if (!admit_slot(S, slot)) return;
            if (!slot->ready) continue;
        }
        std::vector<Request *> batch;
        int kind = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->pending.empty()) return;
                if (!S->pending.empty() && !S->insert_in_flight) {
                    Request *h = S->pending.front();
                    if (h->kind == 0) {
                        int64_t total = 0;
                        while (!S->pending.empty() && S->pending.front()->kind == 0 &&
                               total + S->pending.front()->n <= S->max_batch) {
                            total += S->pending.front()->n;
                            batch.push_back(S->pending.front());
                            S->pending.pop_front();
                        }
                        if (!batch.empty()) {
                            kind = 0;
                            ++S->queries_in_flight;
                            break;
                        }
                    } else if (S->queries_in_flight == 0) {
                        batch.push_back(h);
                        S->pending.pop_front();
                        kind = 1;
                        S->insert_in_flight = true;
                        break;
                    }
                }
                S->cv_work.wait(lk);
            }
        }
        dbl_status st = DBL_OK;
        if (kind == 0) {
            int64_t off = 0;
            for (Request *r : batch) {
                std::memcpy(slot->h_u + off, r->a, sizeof(int32_t) * (size_t)r->n);
                std::memcpy(slot->h_v + off, r->b, sizeof(int32_t) * (size_t)r->n);
                off += r->n;
            }
            cudaMemcpyAsync(slot->d_u, slot->h_u, sizeof(int32_t) * (size_t)off, cudaMemcpyHostToDevice, slot->stream);
            cudaMemcpyAsync(slot->d_v, slot->h_v, sizeof(int32_t) * (size_t)off, cudaMemcpyHostToDevice, slot->stream);
            st = dbl_query_ctx(ix, slot->ctx, slot->d_u, slot->d_v, off, slot->d_ans, nullptr, slot->stream);
            if (!st) {
                cudaMemcpyAsync(slot->h_ans, slot->d_ans, (size_t)off, cudaMemcpyDeviceToHost, slot->stream);
                if (cudaStreamSynchronize(slot->stream) != cudaSuccess) st = DBL_ERR_CUDA;
            }
            if (!st) {
                off = 0;
                for (Request *r : batch) {
                    if (r->ans) std::memcpy(r->ans, slot->h_ans + off, (size_t)r->n);
                    off += r->n;
                }
            }
        } else {
            Request *r = batch[0];
            st = dbl_insert_edges_host(ix, r->a, r->b, r->n, slot->stream);
            if (!st && cudaStreamSynchronize(slot->stream) != cudaSuccess) st = DBL_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const Clock::time_point now = Clock::now();
            for (Request *r : batch) {
                r->status = st;
                r->t_done = now;
                r->done = true;
                const double lat = std::chrono::duration<double>(now - r->t_submit).count();
                if (kind == 0) {
                    S->lat_q.push_back(lat);
                    S->queries_done += (uint64_t)r->n;
                } else {
                    S->lat_i.push_back(lat);
                    S->edges_done += (uint64_t)r->n;
                }
            }
            if (kind == 0) {
                --S->queries_in_flight;
                ++S->batches;
                S->batched_requests += batch.size();
            } else {
                S->insert_in_flight = false;
                ++S->epoch;
            }
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

static double percentile(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t i = (size_t)(p * (double)(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
}

extern "C" {

void dbl_server_default_options(dbl_server_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 4;
    o->max_batch = 1 << 18;
    o->max_pending = 1 << 16;
    o->mem_fraction = 0.5;
    o->max_memory = 0;
}

dbl_status dbl_server_create(dbl_index *ix, const dbl_server_options *opt, dbl_server **out)
{
    if (!ix || !out) return DBL_ERR_INVALID;
    *out = nullptr;
    dbl_server_options o;
    dbl_server_default_options(&o);
    if (opt) o = *opt;
    if (o.slots < 1 || o.max_batch < 1 || o.max_pending < 1 || o.mem_fraction <= 0 || o.mem_fraction > 1 ||
        o.max_memory < 0)
        return dbl::fail(ix, DBL_ERR_INVALID, "server: bad options");
    if (ix->opt.flags & DBL_FLAG_ASYNC) return dbl::fail(ix, DBL_ERR_INVALID, "server: index must not be ASYNC");
    // admission by free HBM: each slot needs its search scratch (the state
    // table, lists, tasks) plus staging for max_batch pairs
    const int64_t W = 1 + ix->wd + 2 * ix->wb;
    const int64_t table = dbl::search_table_slots(ix);
    const int64_t per_slot = table * (32 + 12) + ((int64_t)ix->n_cap + (ix->m + ix->edge_cap) / dbl::kChunk) * 24 +
                             o.max_batch * (int64_t)(4 + 8 * W + 9 + 1) + (64 << 20);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return dbl::fail(ix, DBL_ERR_CUDA, "server: cudaMemGetInfo");
    if ((double)per_slot > (double)free_b * o.mem_fraction || (o.max_memory > 0 && per_slot > o.max_memory))
        return dbl::fail(ix, DBL_ERR_OOM, "server: not enough free device memory for one slot");
    dbl_server *S = new dbl_server();
    S->ix = ix;
    S->max_batch = o.max_batch;
    S->max_pending = o.max_pending;
    S->per_slot = per_slot;
    S->mem_fraction = o.mem_fraction;
    S->max_memory = o.max_memory;
    S->slots.resize(o.slots);
    dbl_status st = slot_setup(S, S->slots[0]);  // the others are admitted by memory when needed
    if (!st) S->ready_slots = 1;
    if (st) {
        S->stop = true;
        dbl_server_destroy(S);
        return dbl::fail(ix, st, "server: slot set-up failed");
    }
    S->t0 = Clock::now();
    for (Slot &sl : S->slots) sl.worker = std::thread(serve_worker, S, &sl);
    *out = S;
    return DBL_OK;
}

dbl_status dbl_server_submit(dbl_server *S, int32_t kind, const int32_t *a_host, const int32_t *b_host, int64_t n,
                             uint8_t *ans_host, uint64_t *ticket)
{
    if (!S || (kind != 0 && kind != 1) || n < 0 || (n > 0 && (!a_host || !b_host)) || !ticket) return DBL_ERR_INVALID;
    if (kind == 0 && n > S->max_batch) return DBL_ERR_INVALID;  // a query request must fit one batch
    Request *r = new Request();
    r->kind = kind;
    r->a = a_host;
    r->b = b_host;
    r->n = n;
    r->ans = ans_host;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int64_t)S->pending.size() >= S->max_pending) {
            delete r;
            return DBL_ERR_BUSY;
        }
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->pending.push_back(r);
        S->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();  // a slot still waiting for memory must not swallow the wake-up
    return DBL_OK;
}

dbl_status dbl_server_wait(dbl_server *S, uint64_t ticket, double *latency_s)
{
    if (!S) return DBL_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return DBL_ERR_INVALID;
    Request *r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    dbl_status st = r->status;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    S->all.erase(it);
    delete r;
    return st;
}

dbl_status dbl_server_cancel(dbl_server *S, uint64_t ticket)
{
    if (!S) return DBL_ERR_INVALID;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) return DBL_ERR_INVALID;
        r = it->second;
        auto q = std::find(S->pending.begin(), S->pending.end(), r);
        if (r->done || q == S->pending.end()) return DBL_ERR_BUSY;  // a slot has it, or it is over
        S->pending.erase(q);
        r->status = DBL_ERR_CANCELLED;
        r->t_done = Clock::now();
        r->done = true;
        ++S->cancelled;
    }
    S->cv_work.notify_all();  // the request may have been holding up the queue head
    S->cv_done.notify_all();
    return DBL_OK;
}

dbl_status dbl_server_drain(dbl_server *S)
{
    if (!S) return DBL_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->pending.empty() && S->queries_in_flight == 0 && !S->insert_in_flight; });
    return DBL_OK;
}

dbl_status dbl_server_report(dbl_server *S, double out[16])
{
    if (!S || !out) return DBL_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    const double el = std::chrono::duration<double>(Clock::now() - S->t0).count();
    for (int i = 0; i < 16; ++i) out[i] = 0;
    out[0] = percentile(S->lat_q, 0.50);
    out[1] = percentile(S->lat_q, 0.99);
    out[2] = percentile(S->lat_i, 0.50);
    out[3] = percentile(S->lat_i, 0.99);
    out[4] = (double)S->queries_done;
    out[5] = (double)S->edges_done;
    out[6] = (double)S->lat_q.size();
    out[7] = (double)S->lat_i.size();
    out[8] = (double)S->slots.size();
    out[9] = el;
    out[10] = (double)S->batches;
    out[11] = (double)S->batched_requests;
    out[12] = (double)S->epoch;
    out[13] = (double)S->cancelled;
    out[14] = (double)S->ready_slots;
    out[15] = (double)S->per_slot;
    return DBL_OK;
}

dbl_status dbl_server_reset_stats(dbl_server *S)
{
    if (!S) return DBL_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_q.clear();
    S->lat_i.clear();
    S->queries_done = S->edges_done = S->batches = S->batched_requests = S->cancelled = 0;
    S->t0 = Clock::now();
    return DBL_OK;
}

void dbl_server_destroy(dbl_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (Slot &sl : S->slots)
        if (sl.worker.joinable()) sl.worker.join();
    for (Slot &sl : S->slots) slot_release(sl);
    for (auto &kv : S->all) delete kv.second;
    delete S;
}

}  // extern "C"
