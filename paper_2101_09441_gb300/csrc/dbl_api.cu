// C-ABI entry points of the DBL library (declared in include/dbl.h).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dbl_internal.cuh"
#include "dbl_persistent.cuh"

namespace dbl {

static thread_local std::string g_build_error;

dbl_status fail(dbl_index *ix, dbl_status st, const std::string &msg)
{
    if (ix) ix->err = msg;
    else g_build_error = msg;
    return st;
}

dbl_status cuda_fail(dbl_index *ix, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ix, DBL_ERR_OOM, m);
    return fail(ix, DBL_ERR_CUDA, m);
}

dbl_status alloc_buf(dbl_index *ix, void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *q = nullptr;
    if (ix->opt.alloc) {
        q = ix->opt.alloc(bytes, (void *)s, ix->opt.ctx);
        if (!q) return fail(ix, DBL_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMallocAsync(&q, bytes, s);
        if (e) {
            cudaGetLastError();
            return fail(ix, DBL_ERR_OOM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        }
    }
    ix->owned.push_back(Buf{q, bytes});
    *p = q;
    return DBL_OK;
}

void free_buf(dbl_index *ix, void *p, cudaStream_t s)
{
    if (!p) return;
    for (size_t i = 0; i < ix->owned.size(); ++i) {
        if (ix->owned[i].p == p) {
            size_t bytes = ix->owned[i].bytes;
            ix->owned[i] = ix->owned.back();
            ix->owned.pop_back();
            if (ix->opt.alloc) ix->opt.free(p, bytes, (void *)s, ix->opt.ctx);
            else cudaFreeAsync(p, s);
            return;
        }
    }
}

dbl_status read_status(dbl_index *ix, cudaStream_t s)
{
    cudaMemcpyAsync(ix->h_pinned + 8, ix->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "synchronize");
    uint32_t st = ix->h_pinned[8];
    if (st) cudaMemsetAsync(ix->d_status, 0, sizeof(uint32_t), s);  // consumed
    if (st == DBL_ERR_TIMEOUT || st == DBL_ERR_CAPACITY) {
        // a device loop gave up or a device buffer overflowed mid-update: labels
        // may be short of the fixpoint, so refuse further use until dbl_restore
        ix->poisoned = true;
        fail(ix, (dbl_status)st, "device loop timed out or overflowed; index poisoned until dbl_restore");
    }
    return (dbl_status)st;
}

void atomic_add_host_stat(dbl_index *ix, int idx, uint64_t v, cudaStream_t)
{
    ix->h_stats[idx] += v;
}

static cudaEvent_t take_event(dbl_index *ix)
{
    if (!ix->ev_free.empty()) {
        cudaEvent_t e = ix->ev_free.back();
        ix->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void tbegin(dbl_index *ix, int kind, cudaStream_t s)
{
    if (!(ix->opt.flags & DBL_FLAG_TIMING)) return;
    if (ix->open_kind >= 0) tend(ix, s);
    dbl_index::TimedRange r{kind, take_event(ix), take_event(ix)};
    cudaEventRecord(r.a, s);
    ix->tranges.push_back(r);
    ix->open_kind = kind;
}

void tend(dbl_index *ix, cudaStream_t s)
{
    if (!(ix->opt.flags & DBL_FLAG_TIMING) || ix->open_kind < 0) return;
    cudaEventRecord(ix->tranges.back().b, s);
    ix->open_kind = -1;
}

static int64_t pow2_at_least(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

dbl_status qfail(dbl_qctx *c, dbl_status st, const std::string &msg)
{
    c->err = msg;
    if (c == c->ix->qc) c->ix->err = msg;
    return st;
}

// Context memory comes from the index's allocator, recorded in the context.
static dbl_status ctx_alloc(dbl_qctx *c, void **p, size_t bytes, cudaStream_t s)
{
    dbl_index *ix = c->ix;
    *p = nullptr;
    bytes = (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
    void *q = nullptr;
    {
        std::lock_guard<std::mutex> lock(ix->alloc_mu);
        if (ix->opt.alloc) {
            q = ix->opt.alloc(bytes, (void *)s, ix->opt.ctx);
        } else if (cudaMallocAsync(&q, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            q = nullptr;
        }
    }
    if (!q) return qfail(c, DBL_ERR_OOM, "query context: allocation of " + std::to_string(bytes) + " bytes failed");
    c->owned.push_back(Buf{q, bytes});
    *p = q;
    return DBL_OK;
}

static void ctx_free(dbl_qctx *c, void *p, cudaStream_t s)
{
    if (!p) return;
    dbl_index *ix = c->ix;
    for (size_t i = 0; i < c->owned.size(); ++i) {
        if (c->owned[i].p != p) continue;
        size_t bytes = c->owned[i].bytes;
        c->owned[i] = c->owned.back();
        c->owned.pop_back();
        std::lock_guard<std::mutex> lock(ix->alloc_mu);
        if (ix->opt.alloc) ix->opt.free(p, bytes, (void *)s, ix->opt.ctx);
        else cudaFreeAsync(p, s);
        return;
    }
}

dbl_status qctx_create(dbl_index *ix, dbl_qctx **out, cudaStream_t s)
{
    dbl_qctx *c = new (std::nothrow) dbl_qctx();
    if (!c) return fail(ix, DBL_ERR_OOM, "query context");
    c->ix = ix;
    dbl_status st;
    if ((st = ctx_alloc(c, (void **)&c->d_counts, 4 * kCntWords, s)) || (st = ctx_alloc(c, (void **)&c->d_status, 16, s))) {
        std::string m = c->err;
        qctx_destroy(c, s);
        return fail(ix, st, m);
    }
    if (cudaMallocHost((void **)&c->h_pinned, 64 * sizeof(uint32_t))) {
        cudaGetLastError();
        qctx_destroy(c, s);
        return fail(ix, DBL_ERR_OOM, "query context: pinned words");
    }
    std::memset(c->h_pinned, 0, 64 * sizeof(uint32_t));
    cudaMemsetAsync(c->d_counts, 0, 4 * kCntWords, s);
    cudaMemsetAsync(c->d_status, 0, 16, s);
    *out = c;
    return DBL_OK;
}

void qctx_destroy(dbl_qctx *c, cudaStream_t s)
{
    if (!c) return;
    while (!c->owned.empty()) ctx_free(c, c->owned.back().p, s);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}

dbl_status ensure_search_scratch(dbl_qctx *c, int64_t q, cudaStream_t s)
{
    dbl_index *ix = c->ix;
    dbl_status st;
    const int64_t W = 1 + ix->wd + 2 * ix->wb;
    if (q > c->und_cap) {
        ctx_free(c, c->und, s);
        ctx_free(c, c->qtab, s);
        ctx_free(c, c->found, s);
        c->und = nullptr;
        c->qtab = nullptr;
        c->found = nullptr;
        c->und_cap = 0;  // a failed allocation below leaves nothing to reuse
        int64_t cap = std::max<int64_t>(q, 1 << 16);
        if ((st = ctx_alloc(c, (void **)&c->und, sizeof(int32_t) * (size_t)cap, s))) return st;
        if ((st = ctx_alloc(c, (void **)&c->qtab, sizeof(uint64_t) * (size_t)(cap + 64) * W, s))) return st;
        if ((st = ctx_alloc(c, (void **)&c->found, sizeof(unsigned long long) * (size_t)(cap / 64 + 2), s)))
            return st;
        c->und_cap = cap;
    }
    if (!c->table) {
        const int64_t slots = search_table_slots(ix);
        // all or nothing: a failure frees what was taken, so the next call starts over
        auto undo = [&](dbl_status err) {
            for (void **p : {(void **)&c->table, (void **)&c->claimed, (void **)&c->slot_list[0],
                             (void **)&c->slot_list[1], (void **)&c->stask, &c->pstate}) {
                ctx_free(c, *p, s);
                *p = nullptr;
            }
            c->table_slots = 0;
            c->stask_cap = 0;
            return err;
        };
        if ((st = ctx_alloc(c, (void **)&c->table, sizeof(SearchSlot) * (size_t)slots, s))) return undo(st);
        if ((st = ctx_alloc(c, (void **)&c->claimed, sizeof(int32_t) * (size_t)slots, s))) return undo(st);
        if ((st = ctx_alloc(c, (void **)&c->slot_list[0], sizeof(int32_t) * (size_t)slots, s))) return undo(st);
        if ((st = ctx_alloc(c, (void **)&c->slot_list[1], sizeof(int32_t) * (size_t)slots, s))) return undo(st);
        cudaMemsetAsync(c->table, 0, sizeof(SearchSlot) * (size_t)slots, s);
        // key = empty (all ones) in every slot: set the key words with a strided memset
        cudaMemset2DAsync(c->table, sizeof(SearchSlot), 0xff, sizeof(unsigned long long), (size_t)slots, s);
        c->table_slots = slots;
        int64_t tcap = (int64_t)ix->n_cap + (ix->m + ix->edge_cap) / kChunk + 4096;
        if ((st = ctx_alloc(c, (void **)&c->stask, sizeof(SearchTask) * (size_t)tcap, s))) return undo(st);
        c->stask_cap = tcap;
        if ((st = ctx_alloc(c, &c->pstate, persist_state_bytes(), s))) return undo(st);
    }
    return DBL_OK;
}

__global__ void k_extract_labels(const uint64_t *rec, int32_t n, int32_t rw, int32_t hs, int32_t wd, int32_t wb,
                                 int packed, int32_t k, uint64_t dlm, uint64_t *dl_in, uint64_t *dl_out,
                                 uint64_t *bl_in, uint64_t *bl_out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *r = rec + (size_t)v * rw;
        if (packed) {  // one word per half: DL below bit k, BL from bit k
            if (dl_in) dl_in[v] = r[0] & dlm;
            if (dl_out) dl_out[v] = r[1] & dlm;
            if (bl_in) bl_in[v] = r[0] >> k;
            if (bl_out) bl_out[v] = r[1] >> k;
            continue;
        }
        for (int w = 0; w < wd; ++w) {
            if (dl_in) dl_in[(size_t)v * wd + w] = r[w];
            if (dl_out) dl_out[(size_t)v * wd + w] = r[hs + w];
        }
        for (int w = 0; w < wb; ++w) {
            if (bl_in) bl_in[(size_t)v * wb + w] = r[wd + w];
            if (bl_out) bl_out[(size_t)v * wb + w] = r[hs + wd + w];
        }
    }
}

}  // namespace dbl

using namespace dbl;

static int hs_for(int words) { return words <= 2 ? 2 : (words <= 4 ? 4 : 8); }

// Label widths of Table 5 (16 .. 256 bits).  Widths below 64 use the low
// bits of one 64-bit word; the rest of the word stays zero.
static bool width_ok(int32_t bits) { return bits == 16 || bits == 32 || bits == 64 || bits == 128 || bits == 256; }

extern "C" {

void dbl_default_options(dbl_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->bfs_words = 16;
    opt->team = 1;
}

static void destroy_impl(dbl_index *ix, cudaStream_t s)
{
    if (!ix) return;
    qctx_destroy(ix->qc, s);
    ix->qc = nullptr;
    for (auto &b : ix->owned) {
        if (ix->opt.alloc) ix->opt.free(b.p, b.bytes, (void *)s, ix->opt.ctx);
        else cudaFreeAsync(b.p, s);
    }
    ix->owned.clear();
    if (ix->h_pinned) cudaFreeHost(ix->h_pinned);
    if (ix->copy_stream) cudaStreamDestroy(ix->copy_stream);
    if (ix->ins_copy_stream) cudaStreamDestroy(ix->ins_copy_stream);
    for (auto &e : ix->ev_stage_used)
        if (e) cudaEventDestroy(e);
    for (auto &e : ix->ev_istage_used)
        if (e) cudaEventDestroy(e);
    for (auto &e : ix->ev_istage_in)
        if (e) cudaEventDestroy(e);
    for (auto &r : ix->tranges) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ix->ev_free) cudaEventDestroy(e);
    delete ix;
}

void dbl_destroy(dbl_index *ix, void *stream)
{
    if (!ix) return;
    drop_insertions(ix);  // queued batches are never applied
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamSynchronize(s);
    destroy_impl(ix, s);
}

dbl_status dbl_build(const dbl_graph *g, const int32_t *landmarks, int32_t k, const int32_t *leaf_buckets,
                     const uint8_t *leaf_roles, int32_t kprime, const dbl_options *opt, void *stream,
                     dbl_index **out)
{
    return dbl::build_index(g, landmarks, k, leaf_buckets, leaf_roles, kprime, opt, stream, out, true);
}

}  // extern "C"

namespace dbl {
// dbl_build, or (labels == false, for dbl_load) the same index with its
// landmark and leaf choices but no labels computed.
dbl_status build_index(const dbl_graph *g, const int32_t *landmarks, int32_t k, const int32_t *leaf_buckets,
                       const uint8_t *leaf_roles, int32_t kprime, const dbl_options *opt, void *stream,
                       dbl_index **out, bool labels)
{
    if (!out) return fail(nullptr, DBL_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g || g->n < 0 || g->m < 0 || g->m >= (1ll << 31) || !g->row_ptr || (g->m > 0 && !g->col))
        return fail(nullptr, DBL_ERR_INVALID, "graph: need n >= 0, 0 <= m < 2^31 and device row_ptr/col");
    if (!width_ok(k) || !width_ok(kprime))
        return fail(nullptr, DBL_ERR_INVALID, "k and kprime must be 16, 32, 64, 128 or 256");
    if (leaf_buckets && !leaf_roles) return fail(nullptr, DBL_ERR_INVALID, "leaf_roles required with leaf_buckets");
    if (opt && ((opt->alloc == nullptr) != (opt->free == nullptr)))
        return fail(nullptr, DBL_ERR_INVALID, "options: alloc and free must be set together");
    if (opt && opt->team && opt->team != 1 && opt->team != 4 && opt->team != 8 && opt->team != 16 && opt->team != 32)
        return fail(nullptr, DBL_ERR_INVALID, "options: team must be 1, 4, 8, 16 or 32");
    if (opt && (opt->landmark_rule < 0 || opt->landmark_rule > 3 || opt->leaf_r < 0))
        return fail(nullptr, DBL_ERR_INVALID, "options: landmark_rule must be 0..3 and leaf_r >= 0");
    if (opt && opt->vertex_capacity >= (1ll << 31))
        return fail(nullptr, DBL_ERR_INVALID, "options: vertex_capacity must be below 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    dbl_index *ix = new (std::nothrow) dbl_index();
    if (!ix) return fail(nullptr, DBL_ERR_OOM, "host allocation");
    dbl_default_options(&ix->opt);
    if (opt) {
        ix->opt = *opt;
        if (!ix->opt.team) ix->opt.team = 1;
        if (!ix->opt.bfs_words) ix->opt.bfs_words = 16;
    }
    cudaGetDevice(&ix->device);
    if (ix->opt.flags & DBL_FLAG_FINE_L2) {
        if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32) != cudaSuccess) cudaGetLastError();
    }
    ix->n = g->n;
    ix->n_cap = (int32_t)std::max<int64_t>(g->n, ix->opt.vertex_capacity);
    ix->m = g->m;
    ix->k = k;
    ix->kp = kprime;
    ix->wd = (k + 63) / 64;
    ix->wb = (kprime + 63) / 64;
    ix->hs = hs_for(ix->wd + ix->wb);
    ix->packed = k + kprime <= 64;  // Table 5's small labels: one word per half, 16-byte records
    if (ix->packed) {
        ix->hs = 1;
        ix->bl_base = k;
        ix->dl_mask = (1ull << k) - 1;
        ix->bl_mask = ((kprime == 64 ? ~0ull : (1ull << kprime) - 1)) << k;
    } else {
        ix->bl_base = 64 * ix->wd;
    }
    ix->rw = 2 * ix->hs;
    ix->edge_cap = ix->opt.edge_capacity > 0 ? ix->opt.edge_capacity : std::max<int64_t>(1 << 20, g->m / 4);
    if (ix->edge_cap > (1ll << 29)) ix->edge_cap = 1ll << 29;  // per-vertex slots then fit in 30 bits
    if (ix->edge_cap + g->m >= (1ll << 31)) ix->edge_cap = (1ll << 31) - 1 - g->m;
    // slots reserved per vertex and direction: a power of two (the capacity is
    // kept as its log2), at least 2, at most 64; none if they would take more
    // than half of the pool's 2^31 addressable entries
    {
        int32_t want = ix->opt.initial_slots == 0 ? 4 : ix->opt.initial_slots;
        int32_t s0 = 0;
        if (want > 0) {
            s0 = 2;
            while (s0 < want && s0 < 64) s0 <<= 1;
        }
        if ((int64_t)s0 * std::max<int64_t>(g->n, ix->opt.vertex_capacity) > (1ll << 30)) s0 = 0;
        ix->slots0 = s0;
    }
    const int64_t reserved_slots = (int64_t)ix->slots0 * std::max<int64_t>(g->n, ix->opt.vertex_capacity);
    if (reserved_slots + 4 * ix->edge_cap + 64 >= (1ll << 31)) ix->edge_cap = ((1ll << 31) - 65 - reserved_slots) / 4;
    ix->pool_cap = reserved_slots + 4 * ix->edge_cap + 64;

    // per-vertex arrays hold n_cap rows (vertex insertion); the base CSR holds the build's n
    const size_t n = (size_t)ix->n_cap, m = (size_t)ix->m, nb = (size_t)ix->n;
    dbl_status st;
    auto A = [&](void **p, size_t bytes) { return alloc_buf(ix, p, bytes, s); };
    if (cudaMallocHost((void **)&ix->h_pinned, 64 * sizeof(uint32_t))) {
        cudaGetLastError();
        destroy_impl(ix, s);
        return fail(nullptr, DBL_ERR_OOM, "pinned host words");
    }
    std::memset(ix->h_pinned, 0, 64 * sizeof(uint32_t));
    ix->front_cap = 2 * ((int64_t)n + (int64_t)(m + ix->edge_cap) / kChunk + 64);
    ix->wpd = ((int64_t)n + 31) / 32 + 1;  // + 1: never zero words
    if ((st = A((void **)&ix->out_ptr, 4 * (nb + 1))) || (st = A((void **)&ix->out_col, 4 * m)) ||
        (st = A((void **)&ix->in_ptr, 4 * (nb + 1))) || (st = A((void **)&ix->in_col, 4 * m)) ||
        (st = A((void **)&ix->vm, sizeof(VMeta) * n)) ||
        (st = A((void **)&ix->pool_out, 4 * (size_t)ix->pool_cap)) ||
        (st = A((void **)&ix->pool_in, 4 * (size_t)ix->pool_cap)) || (st = A((void **)&ix->d_pool_top, 16)) ||
        (st = A((void **)&ix->rec, 8 * n * ix->rw)) || (st = A((void **)&ix->landmarks, 4 * (size_t)k)) ||
        (st = A((void **)&ix->leaf_bucket, 4 * n)) || (st = A((void **)&ix->leaf_role, n)) ||
        (st = A((void **)&ix->mark, 16 * (size_t)ix->wpd)) ||
        (st = A((void **)&ix->front[0], sizeof(FTask) * (size_t)ix->front_cap)) ||
        (st = A((void **)&ix->front[1], sizeof(FTask) * (size_t)ix->front_cap)) || (st = A((void **)&ix->d_counts, 4 * kCntWords)) ||
        (st = A((void **)&ix->d_status, 16)) || (st = A((void **)&ix->d_stats, 8 * 16)) ||
        (st = A((void **)&ix->d_trace, 8 * 64)) ||
        (st = A((void **)&ix->ins_cnt, 8 * n)) ||
        (st = A((void **)&ix->dirty, 4 * (n / 32 + 1))) || (st = A((void **)&ix->d_restore_base, 16))) {
        std::string msg = ix->err;
        destroy_impl(ix, s);
        return fail(nullptr, st, msg);
    }
    cudaMemsetAsync(ix->vm, 0, sizeof(VMeta) * n, s);
    {   // the pools start after the reserved slots of every vertex row
        const int64_t top0[2] = {reserved_slots, reserved_slots};
        cudaMemcpyAsync(ix->d_pool_top, top0, 16, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);  // top0 lives on this stack frame
    }
    cudaMemsetAsync(ix->mark, 0, 16 * (size_t)ix->wpd, s);
    cudaMemsetAsync(ix->d_counts, 0, 4 * kCntWords, s);
    cudaMemsetAsync(ix->d_status, 0, 16, s);
    cudaMemsetAsync(ix->d_stats, 0, 8 * 16, s);
    cudaMemsetAsync(ix->d_trace, 0, 8 * 64, s);
    cudaMemsetAsync(ix->ins_cnt, 0, 8 * n, s);
    ix->dirty_words = (int64_t)(n / 32 + 1);
    cudaMemsetAsync(ix->dirty, 0, 4 * (size_t)ix->dirty_words, s);
    cudaMemsetAsync(ix->d_restore_base, 0xff, 16, s);  // no snapshot yet

    ix->n_build = g->n;
    tbegin(ix, DBL_KERNEL_BUILD_PREP, s);
    if ((st = prep_graph(ix, g, s)) || (st = select_landmarks(ix, landmarks, s)) ||
        (st = select_leaves(ix, leaf_buckets, leaf_roles, s)) || (labels && (st = seed_labels(ix, s))) ||
        (tend(ix, s), labels && (st = build_propagate(ix, s)))) {
        std::string msg = ix->err;
        destroy_impl(ix, s);
        return fail(nullptr, st, msg);
    }
    if ((st = qctx_create(ix, &ix->qc, s))) {
        std::string msg = ix->err;
        destroy_impl(ix, s);
        return fail(nullptr, st, msg);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) {
        destroy_impl(ix, s);
        return cuda_fail(nullptr, e, "build");
    }
    ix->track_dirty = true;  // from here on every change is recorded for restores
    *out = ix;
    return DBL_OK;
}
}  // namespace dbl

extern "C" {

#define DBL_CHECK_IX(ix)                                                                   \
    do {                                                                                   \
        if (!(ix)) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");                 \
        if ((ix)->poisoned) return fail(ix, DBL_ERR_POISONED, "index poisoned by a timeout; dbl_restore it"); \
    } while (0)

// Every call that reads or changes the index other than by a deferred
// insertion first applies the queued insertion batches (DBL_FLAG_DEFER).
#define DBL_FLUSH(ix, s)                                               \
    do {                                                               \
        if (!(ix)->pending.empty()) {                                  \
            const dbl_status flush_st_ = flush_insertions((ix), (s));  \
            if (flush_st_) return flush_st_;                           \
        }                                                              \
    } while (0)

static dbl_status finish(dbl_index *ix, dbl_status st, cudaStream_t s)
{
    if (st) return st;
    if (ix->opt.flags & DBL_FLAG_ASYNC) return DBL_OK;
    return read_status(ix, s);
}

dbl_status dbl_insert_edges(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, void *stream)
{
    DBL_CHECK_IX(ix);
    if (b < 0 || b >= (1ll << 31) || (b > 0 && (!src || !dst))) return fail(ix, DBL_ERR_INVALID, "insert: bad batch");
    cudaStream_t s = (cudaStream_t)stream;
    return finish(ix, insert_edges(ix, src, dst, b, s), s);
}

dbl_status dbl_query(dbl_index *ix, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans, uint8_t *code,
                     void *stream)
{
    DBL_CHECK_IX(ix);
    if (q < 0 || q >= (1ll << 31) || (q > 0 && (!u || !v || !ans))) return fail(ix, DBL_ERR_INVALID, "query: bad batch");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    return finish(ix, query(ix, ix->qc, u, v, q, ans, code, s), s);
}

dbl_status dbl_qctx_create(dbl_index *ix, dbl_qctx **out, void *stream)
{
    if (!ix || !out) return fail(ix, DBL_ERR_INVALID, "qctx_create: NULL argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    dbl_status st = qctx_create(ix, out, s);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    return e ? cuda_fail(ix, e, "qctx_create") : DBL_OK;
}

void dbl_qctx_destroy(dbl_qctx *c, void *stream)
{
    if (!c) return;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamSynchronize(s);
    qctx_destroy(c, s);
    cudaStreamSynchronize(s);
}

dbl_status dbl_query_ctx(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                         uint8_t *code, void *stream)
{
    if (!ix || !c || c->ix != ix) return fail(ix, DBL_ERR_INVALID, "query_ctx: context of another index");
    if (ix->poisoned) return qfail(c, DBL_ERR_POISONED, "index poisoned by a timeout; dbl_restore it");
    if (q < 0 || q >= (1ll << 31) || (q > 0 && (!u || !v || !ans))) return qfail(c, DBL_ERR_INVALID, "query: bad batch");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    return query(ix, c, u, v, q, ans, code, s);
}

const char *dbl_qctx_last_error(const dbl_qctx *c) { return c ? c->err.c_str() : ""; }

static dbl_status ensure_copy_stream(dbl_index *ix, cudaStream_t *cs)
{
    if (*cs) return DBL_OK;
    cudaError_t e = cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking);
    return e ? cuda_fail(ix, e, "copy stream") : DBL_OK;
}

static dbl_status ensure_stage(dbl_index *ix, int64_t chunk, cudaStream_t s)
{
    if (ix->stage_chunk >= chunk) return DBL_OK;
    dbl_status st;
    ix->stage_chunk = 0;  // a failed allocation below leaves nothing to reuse
    for (int b = 0; b < 2; ++b) {
        free_buf(ix, ix->dstage[b], s);
        ix->dstage[b] = nullptr;
        // u, v (int32) + ans, code (uint8) per pair
        if ((st = alloc_buf(ix, (void **)&ix->dstage[b], (size_t)chunk * 10 + 64, s))) return st;
    }
    if ((st = ensure_copy_stream(ix, &ix->copy_stream))) return st;
    for (auto &e : ix->ev_stage_used) {
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) return cuda_fail(ix, cudaGetLastError(), "stage events");
        // (re)allocated buffers: the first uploads wait for everything queued so far
        cudaEventRecord(e, s);
    }
    ix->stage_chunk = chunk;
    return DBL_OK;
}

dbl_status dbl_query_host(dbl_index *ix, const int32_t *u_host, const int32_t *v_host, int64_t q, uint8_t *ans_host,
                          uint8_t *code_host, void *stream)
{
    DBL_CHECK_IX(ix);
    if (q < 0 || q >= (1ll << 31) || (q > 0 && (!u_host || !v_host || !ans_host)))
        return fail(ix, DBL_ERR_INVALID, "query_host: bad batch");
    if (q == 0) return DBL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    // large chunks: each chunk is one label test and one search (whose cost
    // has a fixed part); the upload of the first chunk overlaps earlier work
    const int64_t chunk = std::min<int64_t>(q, 1 << 24);
    dbl_status st = ensure_stage(ix, chunk, s);
    if (st) return st;
    const int64_t nch = (q + chunk - 1) / chunk;
    // A chunk's upload waits only until the buffer's previous query chunk is done
    // with it (ev_stage_used, kept across calls), not for everything queued on the
    // stream: uploads overlap earlier work such as insertions.
    cudaEvent_t ev_in[2];
    for (int b = 0; b < 2; ++b) cudaEventCreateWithFlags(&ev_in[b], cudaEventDisableTiming);
    auto stage_in = [&](int64_t c) {
        const int b = (int)(c & 1);
        const int64_t off = c * chunk, len = std::min(chunk, q - off);
        char *d = (char *)ix->dstage[b];
        cudaStreamWaitEvent(ix->copy_stream, ix->ev_stage_used[b], 0);
        cudaMemcpyAsync(d, u_host + off, 4 * (size_t)len, cudaMemcpyHostToDevice, ix->copy_stream);
        cudaMemcpyAsync(d + 4 * chunk, v_host + off, 4 * (size_t)len, cudaMemcpyHostToDevice, ix->copy_stream);
        cudaEventRecord(ev_in[b], ix->copy_stream);
    };
    stage_in(0);
    for (int64_t c = 0; c < nch && !st; ++c) {
        const int b = (int)(c & 1);
        const int64_t off = c * chunk, len = std::min(chunk, q - off);
        char *d = (char *)ix->dstage[b];
        if (c + 1 < nch) stage_in(c + 1);  // overlaps this chunk's compute (Section 6.6)
        cudaStreamWaitEvent(s, ev_in[b], 0);
        uint8_t *da = (uint8_t *)(d + 8 * chunk), *dc = (uint8_t *)(d + 9 * chunk);
        st = query(ix, ix->qc, (int32_t *)d, (int32_t *)(d + 4 * chunk), len, da, code_host ? dc : nullptr, s);
        if (st) break;
        cudaMemcpyAsync(ans_host + off, da, (size_t)len, cudaMemcpyDeviceToHost, s);
        if (code_host) cudaMemcpyAsync(code_host + off, dc, (size_t)len, cudaMemcpyDeviceToHost, s);
        cudaEventRecord(ix->ev_stage_used[b], s);
    }
    const bool async = (ix->opt.flags & DBL_FLAG_ASYNC) != 0;
    cudaError_t e = async ? cudaGetLastError() : cudaStreamSynchronize(s);
    if (!async) cudaStreamSynchronize(ix->copy_stream);
    for (int b = 0; b < 2; ++b) cudaEventDestroy(ev_in[b]);  // released once the recorded work completes
    if (st) return st;
    if (e) return cuda_fail(ix, e, "query_host");
    return async ? DBL_OK : read_status(ix, s);
}

dbl_status dbl_insert_edges_host(dbl_index *ix, const int32_t *src_host, const int32_t *dst_host, int64_t b,
                                 void *stream)
{
    DBL_CHECK_IX(ix);
    if (b < 0 || b >= (1ll << 31) || (b > 0 && (!src_host || !dst_host)))
        return fail(ix, DBL_ERR_INVALID, "insert_host: bad batch");
    if (b == 0) return DBL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool defer = deferring(ix);  // the batch joins the queue; its staging buffer is held until the flush
    if (!defer) DBL_FLUSH(ix, s);
    dbl_status st;
    if (b > ix->istage_cap) {
        DBL_FLUSH(ix, s);  // queued batches may still read the buffers replaced here
        // stream-ordered frees: after every insertion queued on s (each waited for its upload)
        for (int k = 0; k < ix->istage_n; ++k) {
            free_buf(ix, ix->istage[k], s);
            ix->istage[k] = nullptr;
        }
        ix->istage_cap = 0;
        ix->istage_n = 0;
        const int64_t cap = std::max<int64_t>(b, 1 << 16);
        const int nbuf = (int)std::min<int64_t>(dbl_index::kMaxIStage, std::max<int64_t>(2, (64ll << 20) / (8 * cap)));
        for (int k = 0; k < nbuf; ++k) {
            if ((st = alloc_buf(ix, &ix->istage[k], 8 * (size_t)cap, s))) return st;
            ix->istage_n = k + 1;
        }
        if ((st = ensure_copy_stream(ix, &ix->ins_copy_stream))) return st;
        for (int k = 0; k < nbuf; ++k) {
            for (cudaEvent_t *e : {&ix->ev_istage_used[k], &ix->ev_istage_in[k]})
                if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming))
                    return cuda_fail(ix, cudaGetLastError(), "insertion stage events");
            cudaEventRecord(ix->ev_istage_used[k], s);  // new buffers: first uploads follow what is queued
        }
        ix->istage_cap = cap;
        ix->istage_turn = 0;
    }
    // The buffers in turn: a batch's upload (own copy stream) waits only until
    // the insertion that last read its buffer is done, so uploads run ahead of
    // the insertions (a step of up to istage_n batches uploads all of them
    // before a query upload queued after it); the insertion waits for its own
    // upload.
    const int k = ix->istage_turn;
    ix->istage_turn = (k + 1) % ix->istage_n;
    if (ix->istage_queued[k]) DBL_FLUSH(ix, s);  // the ring came round to a batch still queued
    char *d = (char *)ix->istage[k];
    cudaStream_t cs = ix->ins_copy_stream;
    cudaStreamWaitEvent(cs, ix->ev_istage_used[k], 0);
    cudaMemcpyAsync(d, src_host, 4 * (size_t)b, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(d + 4 * ix->istage_cap, dst_host, 4 * (size_t)b, cudaMemcpyHostToDevice, cs);
    cudaEventRecord(ix->ev_istage_in[k], cs);
    cudaStreamWaitEvent(s, ix->ev_istage_in[k], 0);
    st = insert_edges(ix, (int32_t *)d, (int32_t *)(d + 4 * ix->istage_cap), b, s);
    if (defer && !st) ix->istage_queued[k] = true;  // flush_insertions records its use
    else cudaEventRecord(ix->ev_istage_used[k], s);
    if (st) return st;
    return (ix->opt.flags & DBL_FLAG_ASYNC) ? DBL_OK : read_status(ix, s);
}

dbl_status dbl_labels(dbl_index *ix, uint64_t *dl_in, uint64_t *dl_out, uint64_t *bl_in, uint64_t *bl_out,
                      void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    int64_t blocks = ((int64_t)ix->n + kBlock - 1) / kBlock;
    blocks = std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)num_sms() * 16);
    k_extract_labels<<<(unsigned)blocks, kBlock, 0, s>>>(ix->rec, ix->n, ix->rw, ix->hs, ix->wd, ix->wb,
                                                         ix->packed ? 1 : 0, ix->k, ix->dl_mask, dl_in, dl_out,
                                                         bl_in, bl_out);
    ++ix->launches;
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "labels");
    return finish(ix, DBL_OK, s);
}

dbl_status dbl_selection(dbl_index *ix, int32_t *landmarks, int32_t *leaf_buckets, uint8_t *leaf_roles, void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (landmarks)
        cudaMemcpyAsync(landmarks, ix->landmarks, 4 * (size_t)ix->k, cudaMemcpyDeviceToDevice, s);
    if (leaf_buckets)
        cudaMemcpyAsync(leaf_buckets, ix->leaf_bucket, 4 * (size_t)ix->n, cudaMemcpyDeviceToDevice, s);
    if (leaf_roles) cudaMemcpyAsync(leaf_roles, ix->leaf_role, (size_t)ix->n, cudaMemcpyDeviceToDevice, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "selection");
    return finish(ix, DBL_OK, s);
}

dbl_status dbl_add_vertices(dbl_index *ix, int64_t count, int32_t *first, void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    if (ix->poisoned) return fail(ix, DBL_ERR_POISONED, "index poisoned; dbl_restore first");
    if (count < 0) return fail(ix, DBL_ERR_INVALID, "add_vertices: negative count");
    if ((int64_t)ix->n + count > (int64_t)ix->n_cap)
        return fail(ix, DBL_ERR_CAPACITY, "add_vertices: vertex capacity " + std::to_string(ix->n_cap) + " exceeded");
    if (first) *first = ix->n;
    if (count == 0) return DBL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    const size_t v0 = (size_t)ix->n, c = (size_t)count;
    // the rows may hold a vertex that a restore took away: clear them all
    cudaMemsetAsync(ix->rec + v0 * ix->rw, 0, 8 * c * ix->rw, s);
    init_vmeta_rows(ix, (int32_t)v0, (int32_t)c, s);  // no edges; each row's reserved slots
    cudaMemsetAsync(ix->leaf_bucket + v0, 0xff, 4 * c, s);  // -1: not a leaf
    cudaMemsetAsync(ix->leaf_role + v0, 0, c, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "add_vertices");
    ix->n += (int32_t)count;
    return finish(ix, DBL_OK, s);
}

// The snapshot slot the index equals from now on (see k_restore).
__global__ void k_set_restore_base(uint32_t *base, uint32_t slot) { *base = slot; }

dbl_status dbl_snapshot(dbl_index *ix, int slot, void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    if (slot < 0 || slot >= 4) return fail(ix, DBL_ERR_INVALID, "snapshot slot must be 0..3");
    if (ix->poisoned) return fail(ix, DBL_ERR_POISONED, "cannot snapshot a poisoned index");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    Snapshot &sn = ix->snaps[slot];
    dbl_status st;
    const size_t rec_b = 8 * (size_t)ix->n * ix->rw, meta_b = sizeof(VMeta) * (size_t)ix->n;
    if (!sn.rec.p || !sn.vm.p || !sn.top.p) {  // sized for the vertex capacity: a later snapshot into the slot may hold more vertices
        if ((st = alloc_buf(ix, &sn.rec.p, 8 * (size_t)ix->n_cap * ix->rw, s)) ||
            (st = alloc_buf(ix, &sn.vm.p, sizeof(VMeta) * (size_t)ix->n_cap, s)) ||
            (st = alloc_buf(ix, &sn.top.p, 16, s))) {
            for (void **p : {&sn.rec.p, &sn.vm.p, &sn.top.p}) {  // all or nothing
                free_buf(ix, *p, s);
                *p = nullptr;
            }
            return st;
        }
    }
    cudaMemcpyAsync(sn.rec.p, ix->rec, rec_b, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(sn.vm.p, ix->vm, meta_b, cudaMemcpyDeviceToDevice, s);
    // pool tops stay on the device, so that a restore is all device-to-device
    // copies (and can be captured in a CUDA graph)
    cudaMemcpyAsync(sn.top.p, ix->d_pool_top, 16, cudaMemcpyDeviceToDevice, s);
    // the index now equals this slot: track changes from here
    cudaMemsetAsync(ix->dirty, 0, 4 * (size_t)ix->dirty_words, s);
    k_set_restore_base<<<1, 1, 0, s>>>(ix->d_restore_base, (uint32_t)slot);
    ++ix->launches;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "snapshot");
    sn.edges_stored = ix->edges_stored;
    sn.n = ix->n;
    sn.seq = ++ix->snap_seq;
    sn.valid = true;
    return DBL_OK;
}

// Restore, first kernel: the labels and the adjacency metadata.  If the index
// last equalled this slot (device word *base, set by the snapshot or restore
// that cleared the change bitmap) and no device error is latched, only the
// vertices marked in the change bitmap are copied back (every record or
// metadata write since then marked its vertex); otherwise everything is
// copied (16-byte copies, four in flight per thread), and the frontier
// bitmaps are cleared (they are empty after every complete propagation; an
// aborted one may have left bits behind).  Every block reads *base and
// *status before any block could change them: both are written only by the
// second kernel.  The change bitmap is cleared either way.
__global__ void k_restore(uint4 *rec, const uint4 *rec_snap, int64_t rec_units, uint4 *vm, const uint4 *vm_snap,
                          int64_t vm_units, const uint32_t *base, uint32_t slot, const uint32_t *status, int force_full,
                          uint32_t *dirty, int64_t dirty_words, int32_t n_snap, int rec_row_units, uint32_t *mark,
                          int64_t mark_words)
{
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    const bool full = force_full || *(const volatile uint32_t *)base != slot || *(const volatile uint32_t *)status != 0;
    if (!full) {
        // a warp per bitmap word, a lane per vertex: the word's 32 vertices
        // are adjacent in every array, and the grid's warps walk the words in
        // order, so the pages in use at any time span a window of about
        // (warps x 32) vertices instead of the whole arrays
        const int lane = threadIdx.x & 31;
        const int64_t nwarps = st >> 5;
        for (int64_t w = i0 >> 5; w < dirty_words; w += nwarps) {  // warp-uniform
            const uint32_t d = dirty[w];
            if (!d) continue;
            __syncwarp();
            if (lane == 0) dirty[w] = 0;
            const int64_t x = w * 32 + lane;
            if (!((d >> lane) & 1u) || x >= n_snap) continue;  // vertices added after the snapshot go away
            uint4 r[8], m0, m1;  // a record is 1, 2, 4 or 8 units of 16 bytes
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < rec_row_units) r[u] = __ldcs(rec_snap + x * rec_row_units + u);
            m0 = __ldcs(vm_snap + 2 * x);
            m1 = __ldcs(vm_snap + 2 * x + 1);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < rec_row_units) rec[x * rec_row_units + u] = r[u];
            vm[2 * x] = m0;
            vm[2 * x + 1] = m1;
        }
        return;
    }
    const int64_t total = rec_units + vm_units;
    for (int64_t i = i0; i < total; i += 4 * st) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = i + k * st;
            if (j < total) v[k] = j < rec_units ? __ldcs(rec_snap + j) : __ldcs(vm_snap + (j - rec_units));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t j = i + k * st;
            if (j < total) {
                if (j < rec_units) __stcs(rec + j, v[k]);
                else __stcs(vm + (j - rec_units), v[k]);
            }
        }
    }
    for (int64_t i = i0; i < mark_words; i += st) mark[i] = 0;
    for (int64_t i = i0; i < dirty_words; i += st) dirty[i] = 0;
}

// Restore, second kernel: pool tops, cleared status and counters, and the
// slot the index now equals.
__global__ void k_restore_finish(int64_t *top, const int64_t *top_snap, uint32_t *status, uint32_t *counts,
                                 int ncounts, uint32_t *base, uint32_t slot)
{
    if (threadIdx.x < 2) top[threadIdx.x] = top_snap[threadIdx.x];
    if (threadIdx.x == 0) {
        *status = 0;
        *base = slot;
    }
    for (int i = threadIdx.x; i < ncounts; i += blockDim.x) counts[i] = 0;
}

dbl_status dbl_restore(dbl_index *ix, int slot, void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    if (slot < 0 || slot >= 4 || !ix->snaps[slot].valid) return fail(ix, DBL_ERR_INVALID, "no snapshot in that slot");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    Snapshot &sn = ix->snaps[slot];
    // Snapshots taken after this one name inserted-edge segments in the part
    // of the edge pool (and in the spare room of segments) that insertions
    // after this restore reuse: they are dropped.  Older snapshots stay valid.
    for (Snapshot &o : ix->snaps)
        if (&o != &sn && o.valid && o.seq > sn.seq) o.valid = false;
    const size_t rec_b = 8 * (size_t)sn.n * ix->rw, meta_b = sizeof(VMeta) * (size_t)sn.n;
    // a poisoned index (an aborted update) is always copied back in full
    k_restore<<<(unsigned)num_sms() * 8, kBlock, 0, s>>>(
        (uint4 *)ix->rec, (const uint4 *)sn.rec.p, (int64_t)(rec_b / 16), (uint4 *)ix->vm, (const uint4 *)sn.vm.p,
        (int64_t)(meta_b / 16), ix->d_restore_base, (uint32_t)slot, ix->d_status, ix->poisoned ? 1 : 0, ix->dirty,
        ix->dirty_words, sn.n, ix->rw / 2, ix->mark, 4 * ix->wpd);
    k_restore_finish<<<1, 32, 0, s>>>(ix->d_pool_top, (const int64_t *)sn.top.p, ix->d_status, ix->d_counts,
                                      kCntWords, ix->d_restore_base, (uint32_t)slot);
    ix->launches += 2;
    ix->edges_stored = sn.edges_stored;
    ix->n = sn.n;
    ix->poisoned = false;
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "restore");
    return finish(ix, DBL_OK, s);
}

dbl_status dbl_barrier_probe(dbl_index *ix, int64_t spin_limit, int32_t absent_block, void *stream)
{
    DBL_CHECK_IX(ix);
    if (spin_limit < 1 || spin_limit > (int64_t)kSpinLimit || absent_block < -1 || absent_block >= num_sms())
        return fail(ix, DBL_ERR_INVALID, "barrier_probe: spin_limit must be 1..2^24, absent_block -1..SMs-1");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    dbl_status st = barrier_probe(ix, spin_limit, absent_block, s);
    if (st) return st;
    return read_status(ix, s);  // a wait that ran out: DBL_ERR_TIMEOUT, index poisoned
}

dbl_status dbl_sync(dbl_index *ix, void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    dbl_status st = read_status(ix, s);
    // queries latch their errors in the status word of the default query context
    cudaMemcpyAsync(ix->qc->h_pinned + 8, ix->qc->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "sync");
    const uint32_t q = ix->qc->h_pinned[8];
    if (q) {
        cudaMemsetAsync(ix->qc->d_status, 0, sizeof(uint32_t), s);
        if (q == DBL_ERR_TIMEOUT) ix->poisoned = true;
        if (!st) st = fail(ix, (dbl_status)q, "query: device error (invalid id or search timeout)");
    }
    return st;
}

dbl_status dbl_stats(dbl_index *ix, uint64_t counters[16], void *stream)
{
    if (!ix || !counters) return fail(ix, DBL_ERR_INVALID, "stats: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    unsigned long long *h = (unsigned long long *)(ix->h_pinned + 16);  // 16 words = 8 u64; use two copies
    uint64_t dev[16];
    cudaMemcpyAsync(h, ix->d_stats, 8 * 8, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "stats");
    std::memcpy(dev, h, 64);
    cudaMemcpyAsync(h, ix->d_stats + 8, 8 * 8, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "stats");
    std::memcpy(dev + 8, h, 64);
    for (int i = 0; i < 16; ++i) counters[i] = dev[i] + ix->h_stats[i];
    return DBL_OK;
}

dbl_status dbl_timings(dbl_index *ix, double ms[8], uint64_t launches[8], void *stream)
{
    if (!ix || !ms || !launches) return fail(ix, DBL_ERR_INVALID, "timings: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    tend(ix, s);
    for (int i = 0; i < 8; ++i) {
        ms[i] = 0;
        launches[i] = 0;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "timings");
    for (auto &r : ix->tranges) {
        float t = 0;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < 8) {
            ms[r.kind] += t;
            launches[r.kind] += 1;
        }
        ix->ev_free.push_back(r.a);
        ix->ev_free.push_back(r.b);
    }
    cudaGetLastError();
    ix->tranges.clear();
    return DBL_OK;
}

dbl_status dbl_phase_trace(dbl_index *ix, int64_t out[64], void *stream)
{
    if (!ix || !out) return fail(ix, DBL_ERR_INVALID, "phase_trace: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    DBL_FLUSH(ix, s);
    unsigned long long h[64];
    cudaError_t e = cudaMemcpyAsync(h, ix->d_trace, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "phase_trace");
    const int64_t marks = h[0] < 64 ? (int64_t)h[0] : 63;
    for (int i = 0; i < 64; ++i) out[i] = 0;
    out[0] = marks;
    for (int64_t i = 1; i <= marks; ++i) out[i] = (int64_t)(h[i] - h[1]);
    return DBL_OK;
}

dbl_status dbl_info(const dbl_index *ix, int64_t info[16])
{
    if (!ix || !info) return DBL_ERR_INVALID;
    for (int i = 8; i < 16; ++i) info[i] = 0;
    info[8] = (int64_t)ix->launches;
    info[9] = ix->hs;
    info[0] = ix->n;
    info[10] = ix->n_cap;
    info[1] = ix->k;
    info[2] = ix->kp;
    info[3] = ix->edges_stored;
    info[4] = ix->edge_cap;
    info[5] = ix->m;
    info[6] = ix->rw * 8;
    info[7] = ix->opt.flags;
    return DBL_OK;
}

const char *dbl_last_error(const dbl_index *ix)
{
    if (!ix) return g_build_error.c_str();
    return ix->err.c_str();
}

}  // extern "C"
