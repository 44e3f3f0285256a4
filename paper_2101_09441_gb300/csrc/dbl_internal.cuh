// Internal declarations of the GB300 DBL library (not part of the C ABI).
//
// Device data layout (one GPU, all resident in HBM):
//   rec     uint64 [n][RW]      per-vertex label record, RW = 2*HS words.
//                               words [0, HS): forward half  = DL_in | BL_in | 0-pad
//                               words [HS, 2HS): backward half = DL_out | BL_out | 0-pad
//                               HS = next power of two >= k/64 + kprime/64, so a
//                               half is 16, 32 or 64 bytes and, for k = kprime = 64,
//                               a whole record is one 32-byte DRAM sector.
//   out_col, in_col          base CSR adjacency of Suc and Pre (int32); the
//                            offsets out_ptr / in_ptr are kept for the build.
//   vm      VMeta [n]        per-vertex adjacency metadata, one 32-byte sector:
//                            per direction the base CSR range and the segment
//                            of inserted edges (offset, length, capacity) in an
//                            edge pool, grown by doubling.  Everything a
//                            frontier or insertion step needs about a vertex's
//                            adjacency is one sector.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "dbl.h"

namespace dbl {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 64;     // edges per propagation / search task
constexpr int kBlock = 256;    // threads per block for frontier kernels

// ------------------------------------------------------------ device views
// Adjacency of a vertex in one direction (dir 0 = Suc, 1 = Pre): base CSR
// edges col[start, start + deg), inserted edges pool[off, off + len) in a
// segment of capacity cap (0: none; else a power of two >= 4).  deg and
// log2(cap) share one word, so a base degree must be below 2^kDegBits.
struct VAdj {
    int32_t start;
    uint32_t dc;  // deg | log2(cap) << kDegBits
    int32_t off;
    int32_t len;
};
struct __align__(32) VMeta {
    VAdj d[2];
};
constexpr int kDegBits = 27;

__host__ __device__ __forceinline__ int32_t va_deg(uint32_t dc) { return (int32_t)(dc & ((1u << kDegBits) - 1u)); }
__host__ __device__ __forceinline__ int32_t va_cap(uint32_t dc)
{
    const uint32_t e = dc >> kDegBits;
    return e ? (int32_t)(1u << e) : 0;
}
__host__ __device__ __forceinline__ uint32_t va_dc(int32_t deg, int32_t cap)
{
    uint32_t e = 0;
    while (cap > 1) {
        cap >>= 1;
        ++e;
    }
    return (uint32_t)deg | (e << kDegBits);
}

struct DevGraph {
    int32_t n;
    VMeta *vm;
    const int32_t *out_col, *in_col;
    const int32_t *pool_out, *pool_in;
    uint32_t *dirty;  // vertices whose record or adjacency changed since the last snapshot / restore (NULL: untracked)
};

// Note that x's record or adjacency metadata changed (a bit per vertex; the
// result is unused, so this is a fire-and-forget reduction).
__device__ __forceinline__ void mark_dirty(uint32_t *dirty, int32_t x)
{
    if (dirty) atomicOr(dirty + (x >> 5), 1u << (x & 31));
}

__device__ __forceinline__ VAdj load_vadj(const VMeta *vm, int dir, int32_t x)
{
    const int4 w = __ldcg(reinterpret_cast<const int4 *>(vm + x) + dir);
    VAdj a;
    a.start = w.x;
    a.dc = (uint32_t)w.y;
    a.off = w.z;
    a.len = w.w;
    return a;
}

// Edge range of x: base part [b0, b0+bd) of col, then inserted part [o0, o0+od) of pool.
struct AdjRange {
    int32_t b0, bd, o0, od;
};

__device__ __forceinline__ AdjRange adj_of(const DevGraph &g, int dir, int32_t x)
{
    const VAdj a = load_vadj(g.vm, dir, x);
    return AdjRange{a.start, va_deg(a.dc), a.off, a.len};
}

// degree of x in direction dir, base + inserted
__device__ __forceinline__ int32_t deg_of(const DevGraph &g, int dir, int32_t x)
{
    const AdjRange r = adj_of(g, dir, x);
    return r.bd + r.od;
}

__device__ __forceinline__ int32_t adj_at(const DevGraph &g, int dir, const AdjRange &r, int32_t e)
{
    if (e < r.bd) return __ldg((dir ? g.in_col : g.out_col) + r.b0 + e);
    return __ldcg((dir ? g.pool_in : g.pool_out) + r.o0 + (e - r.bd));
}

// Where the label halves live: half `dir` of vertex x starts at
// rec + x * stride + dir * boff.  The index's records: stride 2*HS, boff HS
// (forward half, then backward half).  A build pass over one direction alone
// runs on an array of that direction's halves: stride HS, boff 0.
struct RecView {
    uint64_t *rec;
    int64_t stride;
    int64_t boff;
};

__device__ __forceinline__ uint64_t *rec_half(const RecView &r, int32_t x, int dir)
{
    return r.rec + (size_t)x * (size_t)r.stride + (dir ? (size_t)r.boff : 0);
}

// Latch the first error code in the device status word.
__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code)
{
    atomicCAS(status, 0u, code);
}

// A whole 32-byte record (both 16-byte halves at k + k' <= 128) in one
// 256-bit load, cached in L2 only: one request for the record's one DRAM
// sector instead of two 16-byte requests.  p must be 32-byte aligned.
template <typename T>
__device__ __forceinline__ void load_rec32(const uint64_t *p, T &w0, T &w1, T &w2, T &w3)
{
    static_assert(sizeof(T) == 8, "64-bit words");
    asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
                 : "l"(p));
}

template <int HS>
__device__ __forceinline__ void load_half(const uint64_t *p, uint64_t (&w)[HS])
{
    if constexpr (HS == 1) {  // packed labels: a half is one word
        w[0] = __ldcg(p);
        return;
    }
#pragma unroll
    for (int i = 0; i < HS; i += 2) {
        ulonglong2 t = __ldcg(reinterpret_cast<const ulonglong2 *>(p + i));
        w[i] = t.x;
        w[i + 1] = t.y;
    }
}

// Propagation task (16 bytes): up to kChunk consecutive edges of v in one
// direction, located when the task is made (the enqueuer has just read v's
// adjacency metadata), so the consumer goes straight to the edge ids: ncol
// edges of the base CSR from col0, then npool inserted edges from pool0.
struct FTask {
    int32_t v;
    uint32_t meta;  // dir << 31 | (chunk == 0) << 30 | ncol << 8 | npool
    int32_t col0;
    int32_t pool0;
};

__device__ __forceinline__ FTask make_ftask(int32_t v, int dir, int32_t chunk, const AdjRange &r)
{
    const int32_t lo = chunk * kChunk, hi = min(r.bd + r.od, lo + kChunk);
    const int32_t cend = min(hi, r.bd);
    const int32_t ncol = cend > lo ? cend - lo : 0;
    const int32_t pstart = max(lo, r.bd);
    const int32_t npool = hi > pstart ? hi - pstart : 0;
    FTask t;
    t.v = v;
    t.meta = ((uint32_t)dir << 31) | (chunk == 0 ? (1u << 30) : 0u) | ((uint32_t)ncol << 8) | (uint32_t)npool;
    t.col0 = r.b0 + lo;
    t.pool0 = r.o0 + (pstart - r.bd);
    return t;
}

__device__ __forceinline__ int task_dir(const FTask &t) { return (int)(t.meta >> 31); }
__device__ __forceinline__ bool task_first(const FTask &t) { return (t.meta >> 30) & 1u; }
__device__ __forceinline__ int32_t task_ncol(const FTask &t) { return (int32_t)((t.meta >> 8) & 0x7fu); }
__device__ __forceinline__ int32_t task_edges(const FTask &t) { return task_ncol(t) + (int32_t)(t.meta & 0x7fu); }

// Edge e (0 <= e < task_edges) of a task, from its resolved location.
__device__ __forceinline__ int32_t task_edge(const DevGraph &g, int dir, int32_t col0, int32_t ncol, int32_t pool0,
                                            int32_t e)
{
    if (e < ncol) return __ldg((dir ? g.in_col : g.out_col) + col0 + e);
    return __ldcg((dir ? g.pool_in : g.pool_out) + pool0 + (e - ncol));
}

__device__ __forceinline__ FTask load_ftask(const FTask *tasks, int64_t t)
{
    const int4 w = __ldcg(reinterpret_cast<const int4 *>(tasks) + t);
    FTask r;
    r.v = w.x;
    r.meta = (uint32_t)w.y;
    r.col0 = w.z;
    r.pool0 = w.w;
    return r;
}

__device__ __forceinline__ void store_ftask(FTask *tasks, int64_t t, const FTask &v)
{
    reinterpret_cast<int4 *>(tasks)[t] = make_int4(v.v, (int)v.meta, v.col0, v.pool0);
}

// Search task: (group, vertex) state slot, chunk, and the query bits to expand.
struct SearchTask {
    int32_t x;
    uint32_t g;
    uint32_t chunk;
    uint32_t pad;
    uint64_t mask;
};

// Search state slot, keyed by (group << 32 | vertex); 32 bytes = one sector.
struct SearchSlot {
    unsigned long long key;
    unsigned long long visit;
    unsigned long long pend;
    uint32_t stamp;
    uint32_t pad;
};

constexpr unsigned long long kEmptyKey = ~0ull;

// ------------------------------------------------------------ host side
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Snapshot {
    bool valid = false;
    uint64_t seq = 0;   // order of the snapshots (a restore drops the ones taken after it)
    int32_t n = 0;      // vertex count at the snapshot (vertices added later go away on restore)
    Buf rec, vm;        // labels; per-vertex adjacency metadata
    Buf top;            // the two pool tops (device)
    int64_t edges_stored = 0;
};

}  // namespace dbl

struct dbl_index {
    int device = 0;
    int32_t n = 0;      // vertices now (grows by dbl_add_vertices)
    int32_t n_cap = 0;  // vertices every per-vertex array is sized for
    int32_t n_build = 0;  // vertices of the base CSR (the build's graph)
    int64_t m = 0;
    int32_t k = 0, kp = 0, wd = 0, wb = 0, hs = 0, rw = 0;
    // packed labels (k + kprime <= 64): a half is one word, DL in bits
    // [0, k), BL in bits [k, k + kprime); otherwise DL fills words [0, wd) and
    // BL words [wd, wd + wb).  bl_base: the bit where BL starts in a half.
    bool packed = false;
    int32_t bl_base = 0;
    uint64_t dl_mask = ~0ull, bl_mask = ~0ull;  // packed: the bits of DL and of BL in the half word
    dbl_options opt{};
    std::string err;
    bool poisoned = false;

    // graph
    int32_t *out_ptr = nullptr, *out_col = nullptr, *in_ptr = nullptr, *in_col = nullptr;
    dbl::VMeta *vm = nullptr;  // [n] adjacency metadata incl. the inserted-edge segments
    int32_t *pool_out = nullptr, *pool_in = nullptr;
    int64_t pool_cap = 0, edge_cap = 0;
    int32_t slots0 = 0;           // inserted-edge slots reserved per vertex and direction at build
    int64_t edges_stored = 0;     // host mirror of inserted edges stored
    int64_t *d_pool_top = nullptr; // [2] device bump pointers (out, in)
    int64_t h_pool_top[2] = {0, 0};

    // labels and selection
    uint64_t *rec = nullptr;
    int32_t *landmarks = nullptr, *leaf_bucket = nullptr;
    uint8_t *leaf_role = nullptr;

    // frontier scratch
    uint32_t *mark = nullptr;  // [2 parities][2 directions][wpd] frontier dedup bitmaps (see dbl_frontier.cuh)
    int64_t wpd = 0;           // bitmap words per direction: ceil(n / 32)
    dbl::FTask *front[2] = {nullptr, nullptr};
    int64_t front_cap = 0;
    uint32_t *d_counts = nullptr;     // small device counters (see kCnt*)

    // insertion scratch
    int32_t *ins_cnt = nullptr;       // [2][n_cap] per-vertex batch counts (zero between calls)
    int32_t *ins_pos = nullptr;       // [2][bcap] per-edge slot in its vertex batch
    int64_t ins_bcap = 0;

    // insertion batches queued under DBL_FLAG_DEFER, applied together by the
    // next call that reads or changes the index otherwise
    struct Pending {
        const int32_t *src, *dst;
        int64_t b;
    };
    std::vector<Pending> pending;
    int64_t pending_edges = 0;

    // query scratch of calls without an explicit context (dbl_query)
    struct dbl_qctx *qc = nullptr;

    // change tracking for restores: a bit per vertex whose record or adjacency
    // metadata changed since the last snapshot or restore, and (device word)
    // the snapshot slot the index then equalled (0xffffffff: none).  A restore
    // to that slot copies back only the marked vertices.
    uint32_t *dirty = nullptr;
    int64_t dirty_words = 0;
    uint32_t *d_restore_base = nullptr;
    bool track_dirty = false;  // off during the build (nothing to restore to yet)

    // the propagation's view of the labels when it is not the index's records
    // (a build pass over one direction's halves); rec == nullptr: the records
    dbl::RecView prop_view{nullptr, 0, 0};
    // the graph the propagation runs over when it is not the index's own (the
    // build's degree-ordered copy); vm == nullptr: the index's graph
    dbl::DevGraph prop_graph{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

    // status, counters
    uint32_t *d_status = nullptr;
    unsigned long long *d_stats = nullptr;  // [16]
    unsigned long long *d_trace = nullptr;  // [64] phase marks of the last persistent launch (DBL_FLAG_TIMING)
    uint32_t *h_pinned = nullptr;     // pinned host words for small readbacks

    // host-buffer staging (dbl_query_host / dbl_insert_edges_host)
    void *dstage[2] = {nullptr, nullptr};  // query host form: double-buffered chunks
    int64_t stage_chunk = 0;
    cudaEvent_t ev_stage_used[2] = {nullptr, nullptr};  // recorded when a query chunk is done with its buffer
    // insertion host form: a ring of its own buffers (kMaxIStage at most, 64 MB
    // together), so query uploads overlap insertions and later batches upload
    // while earlier ones run
    static constexpr int kMaxIStage = 16;
    void *istage[kMaxIStage] = {};
    int istage_n = 0;
    int64_t istage_cap = 0;
    int istage_turn = 0;
    cudaEvent_t ev_istage_used[kMaxIStage] = {};  // recorded when an insertion is done with its buffer
    cudaEvent_t ev_istage_in[kMaxIStage] = {};    // recorded when a buffer's upload is done
    bool istage_queued[kMaxIStage] = {};  // its batch waits in the insertion queue (DBL_FLAG_DEFER)
    cudaStream_t copy_stream = nullptr;      // query uploads
    cudaStream_t ins_copy_stream = nullptr;  // insertion uploads (a FIFO of their own: a query upload
                                             //   does not queue behind uploads that wait for insertions)

    // DBL_FLAG_TIMING: event pairs per kernel class, harvested by dbl_timings
    struct TimedRange {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<TimedRange> tranges;
    std::vector<cudaEvent_t> ev_free;
    int open_kind = -1;

    std::atomic<uint64_t> h_stats[16] = {};  // host-side counters merged into dbl_stats
    std::atomic<uint64_t> launches{0};       // kernels launched by this index
    dbl::Snapshot snaps[4];
    uint64_t snap_seq = 0;
    std::vector<dbl::Buf> owned;      // for teardown
    std::mutex alloc_mu;              // allocations may come from several query contexts
};

// Scratch of one query batch in flight: the undecided list, the search's
// query table, state hash table, slot lists and tasks, plus its own counters,
// status word and pinned read-back words.  Batches on different contexts may
// run concurrently on different streams (the labels are only read); one
// context runs one batch at a time.
struct dbl_qctx {
    dbl_index *ix = nullptr;
    int32_t *und = nullptr;           // undecided query indices
    int64_t und_cap = 0;
    uint64_t *qtab = nullptr;         // per undecided query: u, v, DL_out(u), BL_in(v), BL_out(v)
    unsigned long long *found = nullptr;  // per 64-query group
    dbl::SearchSlot *table = nullptr;
    int64_t table_slots = 0;          // power of two
    int32_t *claimed = nullptr;       // slots claimed in the current wave
    int32_t *slot_list[2] = {nullptr, nullptr};
    dbl::SearchTask *stask = nullptr;
    int64_t stask_cap = 0;
    void *pstate = nullptr;           // device state of the persistent search
    uint32_t *d_counts = nullptr;     // own counter words (kCnt*)
    uint32_t *d_status = nullptr;     // own latched status
    uint32_t *h_pinned = nullptr;     // pinned read-back words
    std::vector<dbl::Buf> owned;
    std::string err;
};

// small device counter slots in d_counts
enum {
    kCntFront0 = 0,     // size of frontier buffer 0
    kCntFront1 = 1,     // size of frontier buffer 1
    kCntUnd = 2,        // undecided queries
    kCntSlots0 = 3,     // search slot list 0
    kCntSlots1 = 4,     // search slot list 1
    kCntTasks = 5,      // search tasks
    kCntClaimed = 6,    // claimed slots
    kCntOverflow = 7,   // search wave overflow flag
    kCntBad = 8,        // the persistent insertion's invalid-id flag (zero between launches)
    kCntGrow = 9,       // the persistent insertion's some-segment-must-grow flag (zero between launches)
    kCntP0 = 10,        // (3 words) persistent propagation level counts
    kCntBarLeft = 13,   // grid barrier: blocks done with the launch
    kCntBarCount = 14,  // (2 words, 8-byte aligned) grid barrier: arrivals, uint64
    kCntWords = 16
};

namespace dbl {

// allocation helpers (dbl_api.cu)
dbl_status alloc_buf(dbl_index *ix, void **p, size_t bytes, cudaStream_t s);
void free_buf(dbl_index *ix, void *p, cudaStream_t s);
dbl_status fail(dbl_index *ix, dbl_status st, const std::string &msg);
dbl_status cuda_fail(dbl_index *ix, cudaError_t e, const char *what);
dbl_status read_status(dbl_index *ix, cudaStream_t s);
dbl_status ensure_search_scratch(dbl_qctx *c, int64_t und, cudaStream_t s);
dbl_status qctx_create(dbl_index *ix, dbl_qctx **out, cudaStream_t s);
void qctx_destroy(dbl_qctx *c, cudaStream_t s);
dbl_status qfail(dbl_qctx *c, dbl_status st, const std::string &msg);
void atomic_add_host_stat(dbl_index *ix, int idx, uint64_t v, cudaStream_t s);
size_t persist_state_bytes();  // dbl_query.cu
// bracket the launches between tbegin and tend (no-op without DBL_FLAG_TIMING)
void tbegin(dbl_index *ix, int kind, cudaStream_t s);
void tend(dbl_index *ix, cudaStream_t s);

// Frontier dedup bitmaps of level parity p: [2 directions][wpd words].
inline uint32_t *mark_of(const dbl_index *ix, int parity)
{
    return ix->mark + (size_t)parity * 2 * (size_t)ix->wpd;
}

// The labels as the propagation sees them.
inline RecView rec_view(const dbl_index *ix)
{
    if (ix->prop_view.rec) return ix->prop_view;
    return RecView{ix->rec, (int64_t)ix->rw, (int64_t)ix->hs};
}

inline DevGraph dev_graph(const dbl_index *ix)
{
    DevGraph g;
    g.n = ix->n;
    g.vm = ix->vm;
    g.out_col = ix->out_col;
    g.in_col = ix->in_col;
    g.pool_out = ix->pool_out;
    g.pool_in = ix->pool_in;
    g.dirty = ix->track_dirty ? ix->dirty : nullptr;
    return g;
}

inline DevGraph prop_graph(const dbl_index *ix) { return ix->prop_graph.vm ? ix->prop_graph : dev_graph(ix); }

// Search states per query context (dbl_options.search_table_log2): at least
// 2n (so one 64-query group always fits), and room for several large searches
// at once on small graphs.
inline int64_t search_table_slots(const dbl_index *ix)
{
    if (ix->opt.search_table_log2 > 0) return 1ll << std::min(ix->opt.search_table_log2, 34);
    const int64_t n = ix->n_cap;
    const int64_t want = std::max<int64_t>(std::max<int64_t>(1 << 16, 2 * n), std::min<int64_t>(64 * n, 1ll << 24));
    int64_t p = 1;
    while (p < want) p <<= 1;
    return p;
}

inline int num_sms()
{
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
    }
    return v;
}

// prep (dbl_prep.cu)
dbl_status prep_graph(dbl_index *ix, const dbl_graph *g, cudaStream_t s);
dbl_status select_landmarks(dbl_index *ix, const int32_t *user, cudaStream_t s);
dbl_status select_top(dbl_index *ix, const int32_t *op, const int32_t *ip, const unsigned long long *keys, int32_t n,
                      int32_t k, int32_t *out, cudaStream_t s);
dbl_status select_leaves(dbl_index *ix, const int32_t *bucket, const uint8_t *role, cudaStream_t s);
dbl_status seed_labels(dbl_index *ix, cudaStream_t s);                 // seeds only
dbl_status build_propagate(dbl_index *ix, cudaStream_t s);             // seed frontier + fixpoint
void init_vmeta_rows(dbl_index *ix, int32_t v0, int32_t c, cudaStream_t s);
dbl_status exclusive_scan_i32(dbl_index *ix, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);

// propagation (dbl_propagate.cu): run the fixpoint from frontier buffer 0
// (count in d_counts[kCntFront0]) until no record changes.
dbl_status propagate(dbl_index *ix, cudaStream_t s);
dbl_status propagate_persistent(dbl_index *ix, cudaStream_t s);
dbl_status propagate_records(dbl_index *ix, uint64_t *rec, int32_t hs, cudaStream_t s);
dbl_status barrier_probe(dbl_index *ix, int64_t spin_limit, int32_t absent, cudaStream_t s);
void launch_seed_frontier(dbl_index *ix, cudaStream_t s, int dirs = 3, const int32_t *renum = nullptr);
// insertion batches are queued and applied as one group at the next reading call
bool deferring(const dbl_index *ix);
dbl_status build_index(const dbl_graph *g, const int32_t *landmarks, int32_t k, const int32_t *leaf_buckets,
                       const uint8_t *leaf_roles, int32_t kprime, const dbl_options *opt, void *stream,
                       dbl_index **out, bool labels);  // vertices with a non-zero half (dirs: bit 0 forward, bit 1 backward)

// insertion (dbl_insert.cu)
dbl_status insert_edges(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, cudaStream_t s);
dbl_status insert_edges_core(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, int32_t *pos_out,
                             int32_t *pos_in, cudaStream_t s);
dbl_status flush_insertions(dbl_index *ix, cudaStream_t s);  // apply the queued batches (DBL_FLAG_DEFER)
void drop_insertions(dbl_index *ix);                          // forget them (the index is destroyed)

// query (dbl_query.cu)
dbl_status query(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                 uint8_t *code, cudaStream_t s);

}  // namespace dbl
