/*
 * dbl.h -- C ABI of the GB300 DBL reachability index.
 *
 * DBL (arXiv 2101.09441) answers reachability queries q(u, v) on a directed
 * graph that only gains edges, with two bitset labels per vertex and
 * direction:
 *   DL_in(x)  = landmarks that reach x,   DL_out(x) = landmarks x reaches
 *               (Definition 1, Section 4.1);
 *   BL_in(x)  = hash buckets of zero in-degree leaves that reach x,
 *   BL_out(x) = hash buckets of zero out-degree leaves x reaches
 *               (Definition 2 and the hashing paragraph, Section 4.1; with
 *               dbl_options.leaf_r, also every vertex with M <= leaf_r,
 *               Section 6).
 * Reachability is reflexive: Des(u) and Anc(u) contain u (Table 1).
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers unless the name ends in _host.
 *     They are borrowed: the caller keeps them alive until the stream has
 *     passed the call.  Calls are ordered on `stream` (a cudaStream_t; NULL
 *     means the legacy default stream).
 *   - Vertex ids are int32 in [0, n), n growing by dbl_add_vertices.  Labels
 *     are uint64 words: landmark slot
 *     i is word i/64 bit i%64, bucket b is word b/64 bit b%64.
 *   - An invalid argument is reported as DBL_ERR_INVALID before any state
 *     changes.  Running out of the index's edge or vertex capacity is
 *     DBL_ERR_CAPACITY, with the index unchanged.  A device loop that exceeds its iteration
 *     bound is DBL_ERR_TIMEOUT and leaves the index poisoned (every later
 *     call returns DBL_ERR_POISONED) until dbl_restore.
 *   - The index owns all of its device memory, obtained through
 *     dbl_options.alloc/free (default: cudaMallocAsync/cudaFreeAsync).
 *   - Unless DBL_FLAG_ASYNC is set, each call synchronises `stream` before it
 *     returns, so its status covers the device work.  With DBL_FLAG_ASYNC,
 *     device-side errors latch in the index and are returned by dbl_sync.
 *
 * Nothing here is thread-safe per index: one host thread drives an index.
 */
#ifndef DBL_H
#define DBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbl_index dbl_index;

typedef enum {
    DBL_OK = 0,
    DBL_ERR_INVALID = 1,  /* bad argument or id; nothing changed */
    DBL_ERR_OOM = 2,      /* allocation failed; nothing changed */
    DBL_ERR_CUDA = 3,     /* CUDA runtime error; see dbl_last_error */
    DBL_ERR_TIMEOUT = 4,  /* a device loop exceeded its bound; index poisoned */
    DBL_ERR_CAPACITY = 5, /* inserted-edge capacity exhausted; nothing changed */
    DBL_ERR_BUSY = 6,     /* the serving engine refused admission */
    DBL_ERR_POISONED = 7, /* an earlier timeout poisoned the index */
    DBL_ERR_CANCELLED = 8, /* the serving engine dropped the request before it ran */
    DBL_ERR_IO = 9         /* a file could not be written or read (dbl_save, dbl_load) */
} dbl_status;

/* Deciding rule of a query, in the order of Algorithm 2. */
enum {
    DBL_CODE_UNDECIDED = 0,
    DBL_CODE_SELF = 1,    /* u == v: true (reflexive reachability, Table 1) */
    DBL_CODE_DL = 2,      /* DL_out(u) and DL_in(v) intersect: true (Lemma 1) */
    DBL_CODE_BL = 3,      /* BL containment fails: false (Lemma 2) */
    DBL_CODE_THM1 = 4,    /* DL_out(v) and DL_in(u) intersect: false (Theorem 1) */
    DBL_CODE_THM2 = 5,    /* u or v shares an SCC with a landmark: false (Theorem 2) */
    DBL_CODE_BFS_POS = 6, /* pruned search reached v: true (Algorithm 2) */
    DBL_CODE_BFS_NEG = 7  /* pruned search exhausted: false (Algorithm 2) */
};

/* Option flags. */
enum {
    DBL_FLAG_ASYNC = 1,      /* do not synchronise at the end of each call */
    DBL_FLAG_PERSISTENT = 2, /* run frontier loops in one persistent launch */
    DBL_FLAG_TIMING = 4,     /* bracket kernels with CUDA events (dbl_timings) */
    DBL_FLAG_FINE_L2 = 8,    /* at build, set the CUDA context's maximum L2 fetch
                                granularity to 32 bytes (cudaLimitMaxL2FetchGranularity):
                                label records are gathered 32 random bytes at a time.
                                The limit is per context: it applies to every kernel
                                of the process until changed. */
    DBL_FLAG_DEFER = 16      /* with PERSISTENT and ASYNC: dbl_insert_edges only
                                queues the batch; the queued batches are applied
                                together, in one launch, by the next call that reads
                                or changes the index otherwise (a query, labels,
                                stats, a snapshot, a restore, dbl_sync, ...) or when
                                32 are queued.  Each query observes exactly the
                                insertions queued before it, and the labels equal
                                those of any one-by-one order (the unique least
                                fixpoint).  The edge arrays must stay valid until
                                then; an invalid id in any queued batch rejects the
                                whole group (reported by dbl_sync). */
};

/* Kernel classes reported by dbl_timings. */
enum {
    DBL_KERNEL_PROPAGATE = 0,     /* label propagation levels (build and repair) */
    DBL_KERNEL_QUERY_LABEL = 1,   /* label test of every query pair */
    DBL_KERNEL_SEARCH_EXPAND = 2, /* pruned-search expansion levels */
    DBL_KERNEL_SEARCH_OTHER = 3,  /* search set-up, task build, answers, clearing */
    DBL_KERNEL_INSERT_APPEND = 4, /* validation and adjacency append */
    DBL_KERNEL_INSERT_SEED = 5,   /* repair seeds */
    DBL_KERNEL_BUILD_PREP = 6,    /* transpose, selection, seeding */
    DBL_KERNEL_OTHER = 7
};

/* Directed graph G as CSR of out-edges (Suc), device pointers (Section 2).
 * row_ptr[n+1] non-decreasing from 0 to m; col[m] in [0, n).  Self-loops and
 * duplicate edges are allowed and change no label. */
typedef struct {
    int32_t n;
    int64_t m; /* must be < 2^31 */
    const int32_t *row_ptr;
    const int32_t *col;
} dbl_graph;

/* Device allocator; `stream` is the cudaStream_t of the calling operation. */
typedef void *(*dbl_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dbl_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct {
    dbl_alloc_fn alloc; /* NULL: cudaMallocAsync on the call's stream */
    dbl_free_fn free;   /* must be set iff alloc is set */
    void *ctx;
    int64_t edge_capacity; /* inserted edges the index can hold over its life;
                              0: max(2^20, m/4); at most 2^29 (larger values
                              are clamped) */
    int32_t flags;         /* DBL_FLAG_* */
    int32_t bfs_words;     /* 64-query words per search wave (1..64); 0: 16 */
    int32_t team;          /* lanes per expansion task (4, 8, 16, 32), or 1:
                              one task per lane with the warp walking its
                              tasks' edges 32 at a time; 0: 1 */
    int32_t query_unroll;  /* query pairs per lane group in the label test (1, 2,
                              4); 0: 2 for 32-byte records, 4 for wider ones */
    int32_t search_first_log2; /* a search wave first hashes its states into
                              the first 2^x slots of its table (clamped to the
                              table); a wave that overflows them is rerun over
                              the whole table, and one that overflows the whole
                              table is rerun in halves; 0: 22 */
    int32_t landmark_rule; /* ranking of the landmarks chosen when dbl_build gets
                              none (Section 6, Table 3): 0 = |Pre(u)| * |Suc(u)|
                              (Section 4.1), 1 = max(|Pre|, |Suc|) (A),
                              2 = min (B), 3 = |Pre| + |Suc| (C); ties by id */
    int64_t leaf_r;        /* leaves chosen when dbl_build gets none: every u
                              with M(u) = |Pre(u)| * |Suc(u)| <= leaf_r
                              (Section 6); with M(u) = 0 the roles of
                              Definition 2, otherwise both BL_in and BL_out;
                              0: the zero-degree leaves of Definition 2 */
    int64_t vertex_capacity; /* vertices the index can hold over its life
                              (dbl_add_vertices); 0 or less than n: n; must
                              be below 2^31 */
    int32_t initial_slots; /* inserted-edge slots reserved per vertex and
                              direction at build (rounded up to a power of two,
                              at most 64): an insertion batch whose endpoints
                              all still have room appends, seeds and enqueues
                              in one grid-wide phase; 0: 4; negative: none
                              (segments are made at the first insertion).
                              Costs 8 bytes per slot and vertex; dropped when
                              the pool would not fit 2^31 entries */
    int32_t build_split;   /* label build: 1 propagates the two directions one
                              after the other, each over an array of its own
                              halves (fewer address-translation misses on large
                              graphs); -1 both together over the records; 0:
                              split when the records exceed 256 MB */
    int32_t build_order;   /* label build: 1 propagates over a copy of the graph
                              renumbered in groups of equal log2(in + out
                              degree), largest first (the records of the
                              vertices most edges end at share cache lines and
                              pages); -1 in id order; 0: renumbered when the
                              records exceed 256 MB.  Same labels either way.
                              Costs a copy of the graph (8 B per edge, 40 B per
                              vertex) during the build */
    int32_t search_table_log2; /* 32-byte search states per query context:
                              2^x (a lone 64-query group whose search needs
                              more fails with DBL_ERR_CAPACITY); 0: the larger of
                              2n and min(64n, 2^24), rounded up to a power of
                              two (n: the vertex capacity) */
} dbl_options;

/* Fill *opt with the defaults above. */
void dbl_default_options(dbl_options *opt);

/*
 * Build the index for G (Algorithm 1 and the BL construction of Section 4.1).
 *   landmarks[k]   landmark of slot i, or -1 for an empty slot; NULL: the
 *                  top-k vertices by M(u) = |Pre(u)| * |Suc(u)| (Section 4.1,
 *                  landmark heuristic), or by the ranking landmark_rule of the
 *                  options picks, ties by smaller id.
 *   k              16, 32, 64, 128 or 256 (the label sizes of Table 5;
 *                  below 64 the low k bits of one 64-bit word).
 *   leaf_buckets[n] bucket in [0, kprime) of a leaf, -1 for a non-leaf;
 *                  NULL: zero in-degree vertices seed BL_in and zero
 *                  out-degree vertices seed BL_out (Definition 2; with
 *                  options leaf_r > 0 also every u with 0 < M(u) <= leaf_r,
 *                  seeding both), bucket
 *                  h(v) = floor(frac(v * 0x9E3779B97F4A7C15 / 2^64) * kprime)
 *                  (Fibonacci hashing; the paper leaves h open).
 *   leaf_roles[n]  bit0: seeds BL_in, bit1: seeds BL_out; required when
 *                  leaf_buckets is given, ignored otherwise.
 *   kprime         16, 32, 64, 128 or 256, as k.
 * Landmarks and leaf roles are frozen at build; later insertions keep them.
 * The graph arrays are copied; *out receives the new index.
 */
dbl_status dbl_build(const dbl_graph *g, const int32_t *landmarks, int32_t k,
                     const int32_t *leaf_buckets, const uint8_t *leaf_roles, int32_t kprime,
                     const dbl_options *opt, void *stream, dbl_index **out);

/*
 * Insert b edges (src[i], dst[i]) and repair every label (Algorithm 3, its
 * DL_out mirror and the BL update of Section 5).  The batch is applied as a
 * whole; the labels equal those of any one-by-one order and of a rebuild on
 * the final graph with the same landmarks and leaves.  Self-loops are
 * ignored; duplicates are stored and change nothing.
 */
dbl_status dbl_insert_edges(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b,
                            void *stream);

/*
 * Answer q queries q(u[i], v[i]) (Algorithm 2): ans[i] = 1 iff u[i] reaches
 * v[i]; code[i] (may be NULL) = the DBL_CODE_* rule that decided it.  Pairs the
 * labels leave open run a bit-parallel pruned search, 64 queries per word.
 */
dbl_status dbl_query(dbl_index *ix, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                     uint8_t *code, void *stream);

/*
 * dbl_insert_edges without any memory allocation.  (The paper has no
 * counterpart: this is an interface for callers that cannot allocate.)
 *
 * dbl_insert_edges may allocate per-edge scratch (8 bytes per edge) from the
 * index's allocator when a batch is larger than any before it.  Callers whose
 * device memory is already fully handed to their own pool allocator, or that
 * must not wait on an allocator in the middle of a latency-bound loop, cannot
 * allow that.  This variant takes the scratch from a fixed 8 MiB array in the
 * library's device memory instead (every GPU that loads the library holds it
 * until the process exits); everything else it touches was allocated by
 * dbl_build.  Same arguments, results and errors as dbl_insert_edges, plus:
 *   - b > 1,048,576 edges is rejected with DBL_ERR_INVALID (split the batch);
 *   - the device holding the index must be the current device;
 *   - the first call on a device looks up the array's device address (a
 *     cudaGetSymbolAddress, which allocates nothing); make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process and is valid only in the context that was current at that
 *     first call: after a cudaDeviceReset, do not call this entry point;
 *   - all calls in the process share the one array: calls whose device work
 *     overlaps (on different streams, or on different indexes of the same
 *     device) race on it and must be ordered by the caller.  Each call writes
 *     every scratch entry it reads, so nothing left by an earlier call is used.
 */
dbl_status dbl_insert_edges_noalloc(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b,
                                    void *stream);

/* Host-buffer forms: copy inputs from host memory (pinned or pageable) to
 * the device, run the call, and copy results back, in overlapped chunks
 * (the transfer overlap of Section 6.6).  Synchronous, unless the index was
 * built with DBL_FLAG_ASYNC: then the call returns once its copies and
 * kernels are queued on `stream`, and the host buffers must stay valid and
 * unchanged (and the answers are ready) only after dbl_sync or a
 * synchronisation of `stream`; errors latch as in the other calls. */
dbl_status dbl_query_host(dbl_index *ix, const int32_t *u_host, const int32_t *v_host, int64_t q,
                          uint8_t *ans_host, uint8_t *code_host, void *stream);
dbl_status dbl_insert_edges_host(dbl_index *ix, const int32_t *src_host, const int32_t *dst_host,
                                 int64_t b, void *stream);

/* Copy labels out as [n][k/64] (DL) and [n][kprime/64] (BL) uint64; any
 * pointer may be NULL. */
dbl_status dbl_labels(dbl_index *ix, uint64_t *dl_in, uint64_t *dl_out, uint64_t *bl_in,
                      uint64_t *bl_out, void *stream);

/* Copy out the frozen selection: landmarks[k], leaf_buckets[n], leaf_roles[n]
 * (device pointers, any may be NULL). */
dbl_status dbl_selection(dbl_index *ix, int32_t *landmarks, int32_t *leaf_buckets,
                         uint8_t *leaf_roles, void *stream);

/*
 * Vertex insertion (Section 1: the graph grows by new edges and new
 * vertices).  Appends `count` isolated vertices with ids n .. n + count - 1
 * (*first, may be NULL, receives n): empty labels (they reach and are reached
 * by nothing; they are neither landmarks nor leaves, since both sets are
 * frozen at build) and no edges.  Later insertions and queries may name them.
 * DBL_ERR_CAPACITY if n + count exceeds the vertex capacity, with the index
 * unchanged.  The new rows are cleared on `stream`; the vertex count is host
 * state, so a CUDA graph captured earlier keeps validating ids against the
 * count it was captured with.  A restore returns to the snapshot's vertex
 * count.
 */
dbl_status dbl_add_vertices(dbl_index *ix, int64_t count, int32_t *first, void *stream);

/* Save / restore labels and inserted adjacency in snapshot slot 0..3
 * (device-to-device copies on `stream`).  dbl_restore clears a poisoned index and
 * returns to the snapshot's vertex count.  A restore drops every snapshot
 * taken after the restored one (insertions after the restore reuse the part
 * of the edge pool those snapshots name); older snapshots stay valid.  A
 * captured restore does not drop them when the graph is replayed: after a
 * replay, restore only to the captured slot or to older ones. */
dbl_status dbl_snapshot(dbl_index *ix, int slot, void *stream);
dbl_status dbl_restore(dbl_index *ix, int slot, void *stream);

/* Wait for `stream` and return the first error latched on the device. */
dbl_status dbl_sync(dbl_index *ix, void *stream);

/*
 * Check of the bounded waits (diagnostic; the paper has no counterpart).  One
 * cooperative launch of one block per SM on the index's grid-barrier words:
 * every block but absent_block meets at one barrier, and a block whose wait
 * polls more than spin_limit (1 .. 2^24) times gives up.  absent_block = -1:
 * every block arrives and the call returns DBL_OK.  absent_block in
 * [0, SMs): that block never arrives, the waits run out, and the call returns
 * DBL_ERR_TIMEOUT with the index poisoned (as after any device loop that gave
 * up) until dbl_restore; every block still ends, and the barrier words are
 * reset for the next launch.  Synchronous; labels and graph are untouched.
 */
dbl_status dbl_barrier_probe(dbl_index *ix, int64_t spin_limit, int32_t absent_block, void *stream);

/* Restores and change tracking: dbl_restore copies back only the vertices
 * whose record or adjacency changed since the last dbl_snapshot or
 * dbl_restore when its slot is the one the index then equalled, and
 * everything otherwise (also after a timeout); the device decides, so a
 * captured restore stays correct when later snapshots change the slot the
 * index equals. */

/*
 * Counters since build (synchronises `stream`):
 *  [0..7]  queries decided per DBL_CODE_*     [8]  frontier levels run
 *  [9]     expansion tasks                    [10] edges relaxed
 *  [11]    inserted edges applied             [12] insertions skipped (u reached v)
 *  [13]    self-loops ignored                 [14] search waves
 *  [15]    inserted edges stored
 */
dbl_status dbl_stats(dbl_index *ix, uint64_t counters[16], void *stream);

/*
 * Phase trace of the index's last persistent launch (insertion, label
 * propagation, or the pruned search of a query batch on the index's own
 * context; recorded only when the index was built with DBL_FLAG_TIMING).
 * out[0] = number of marks m (<= 63); out[1..m] = nanoseconds since the launch
 * began (%globaltimer of block 0) at the start, after each grid barrier, and at
 * the end.  An insertion launch's barriers follow its phases: validate +
 * count, seed + grow, write + enqueue, then one per propagation level.
 * Synchronises `stream`.  Diagnostic only: the paper has no counterpart.
 */
dbl_status dbl_phase_trace(dbl_index *ix, int64_t out[64], void *stream);

/* With DBL_FLAG_TIMING: device time (ms, from CUDA events recorded on the
 * launching stream) and launch count per DBL_KERNEL_* class since the last
 * call; synchronises `stream`.  Without the flag both arrays are zero. */
dbl_status dbl_timings(dbl_index *ix, double ms[8], uint64_t launches[8], void *stream);

/* Facts about the index: [0] n, [1] k, [2] kprime, [3] inserted edges stored,
 * [4] edge capacity, [5] base edges m, [6] label record bytes per vertex,
 * [7] option flags, [8] kernels launched so far, [9] words per record half,
 * [10] vertex capacity; [11..15] zero. */
dbl_status dbl_info(const dbl_index *ix, int64_t info[16]);

/*
 * Autotuner: time the sample insertion batch (src, dst, b) followed by the
 * sample query batch (u, v, q; answers to ans) under each frontier schedule
 * -- team widths 1, 4, 8, 16, 32 (dbl_options.team) and
 * level-by-level or persistent propagation -- each `trials` times from the
 * same snapshot (slot 3 is overwritten), and keep the fastest in the index's
 * options.  The index's labels and graph are restored afterwards.
 * report (may be NULL, else 16 doubles) receives [0..9] the fastest trial's ms per
 * candidate (level-by-level teams 1, 4, 8, 16, 32, then persistent teams
 * 1..32), [10] best team, [11] 1 if persistent, [12] best ms, [13..15] the
 * fastest ms of the query batch alone under the chosen schedule with 1, 2
 * and 4 label-test pairs per lane group (dbl_options.query_unroll; the
 * fastest is kept).  DBL_FLAG_ASYNC/TIMING are off during the trials and
 * restored after.  Synchronous.
 */
dbl_status dbl_autotune(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, const int32_t *u,
                        const int32_t *v, int64_t q, uint8_t *ans, int32_t trials, double *report, void *stream);
/* Apply a schedule directly (e.g. one cached from dbl_autotune): team width
 * 1, 4, 8, 16 or 32; persistent != 0 sets DBL_FLAG_PERSISTENT; query_unroll
 * 1, 2 or 4 label-test pairs per lane group (0 keeps the current value). */
dbl_status dbl_set_schedule(dbl_index *ix, int32_t team, int32_t persistent, int32_t query_unroll);

/* ---------------------------------------------------------------------------
 * Concurrent query batches.  A query context holds the scratch of one query
 * batch in flight (undecided list, search state); batches on different
 * contexts may run at the same time on different streams and host threads,
 * as long as no insertion runs meanwhile (queries only read the labels).
 * dbl_query uses the index's own context.  Explicit contexts always use the
 * per-level search (no cooperative launch).
 * ------------------------------------------------------------------------- */
typedef struct dbl_qctx dbl_qctx;
dbl_status dbl_qctx_create(dbl_index *ix, dbl_qctx **out, void *stream);
void dbl_qctx_destroy(dbl_qctx *c, void *stream);
/* dbl_query on context c; synchronous; errors are also in dbl_qctx_last_error. */
dbl_status dbl_query_ctx(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                         uint8_t *code, void *stream);
const char *dbl_qctx_last_error(const dbl_qctx *c);

/* ---------------------------------------------------------------------------
 * Serving engine (continuous batching over one resident index).  Requests
 * are query batches (kind 0: pairs a[i], b[i], answers to ans) or insertion
 * batches (kind 1: edges a[i] -> b[i]) in HOST memory, which the caller keeps
 * alive until dbl_server_wait returns for the ticket.  Admission is in arrival
 * order; consecutive queued queries are packed into one device batch of at
 * most max_batch pairs on a free slot, so several batches overlap on the GPU;
 * an insertion waits until no query batch is in flight and every request
 * behind it waits for it, so each request observes exactly the insertions
 * submitted before it (the labels change only at these epoch boundaries).
 * Admission by memory: a slot's device scratch (a query context sized for
 * max_batch pairs, and staging) is allocated when the slot is first needed,
 * and only if it then fits in mem_fraction of the device's free memory
 * (cudaMemGetInfo, read at that moment); until then requests wait for the
 * slots that have memory.  The first slot is set up at creation
 * (DBL_ERR_OOM if it does not fit).  Submit returns
 * DBL_ERR_BUSY when max_pending requests are queued.  The index must not use
 * DBL_FLAG_ASYNC and must not be used directly while a server runs on it.
 * ------------------------------------------------------------------------- */
typedef struct dbl_server dbl_server;
typedef struct {
    int32_t slots;        /* worker slots (streams); default 4 */
    int64_t max_batch;    /* pairs per device batch; default 2^18 */
    int64_t max_pending;  /* queued requests before DBL_ERR_BUSY; default 2^16 */
    double mem_fraction;  /* a slot is admitted when its scratch fits in this share
                             of the device's free memory at that moment; default 0.5 */
    int64_t max_memory;   /* and when all admitted slots together stay within this
                             many device bytes; 0: no such limit (default) */
} dbl_server_options;
void dbl_server_default_options(dbl_server_options *o);
dbl_status dbl_server_create(dbl_index *ix, const dbl_server_options *opt, dbl_server **out);
dbl_status dbl_server_submit(dbl_server *s, int32_t kind, const int32_t *a_host, const int32_t *b_host, int64_t n,
                             uint8_t *ans_host, uint64_t *ticket);
/* Block until the request is done; returns its status and latency (s);
 * DBL_ERR_CANCELLED for a cancelled request. */
dbl_status dbl_server_wait(dbl_server *s, uint64_t ticket, double *latency_s);
/* Cancel a request that no slot has taken yet: it is dropped from the queue
 * (its answers are not written; a cancelled insertion is never applied, so
 * later requests do not observe it) and dbl_server_wait returns
 * DBL_ERR_CANCELLED for it.  DBL_ERR_BUSY if it is already running or done,
 * DBL_ERR_INVALID for an unknown ticket.  (Request cancellation is part of
 * serving; the paper has no counterpart.) */
dbl_status dbl_server_cancel(dbl_server *s, uint64_t ticket);
dbl_status dbl_server_drain(dbl_server *s);
/* [0] query p50 s, [1] query p99 s, [2] insertion p50 s, [3] insertion p99 s,
 * [4] pairs answered, [5] edges inserted, [6] query requests, [7] insertion
 * requests, [8] slots, [9] seconds since creation or reset, [10] device
 * query batches, [11] query requests in them, [12] insertion epochs,
 * [13] requests cancelled, [14] slots admitted (with scratch), [15] device
 * bytes per slot. */
dbl_status dbl_server_report(dbl_server *s, double out[16]);
dbl_status dbl_server_reset_stats(dbl_server *s);
void dbl_server_destroy(dbl_server *s);

/* ---------------------------------------------------------------------------
 * Learned landmark scorer.  The paper ranks landmarks by M(u) = |Pre(u)| *
 * |Suc(u)| (Section 4.1; Table 3 compares other rankings) and notes that the
 * best choice is NP-hard.  These calls score vertices with a 16-128-128-1 ReLU
 * network instead; answers stay exact for any landmark set (Lemma 1), only
 * how many pairs the DL test decides changes.  Build a new index with
 * dbl_build(landmarks = the selected vertices) to use the result.
 * ------------------------------------------------------------------------- */

typedef struct dbl_mlp dbl_mlp;

/* Number of network parameters and their order in a flat float vector:
 * W1 [16][128] (input x hidden, row-major), b1 [128], W2 [128][128], b2 [128],
 * w3 [128], b3 [1]. */
#define DBL_MLP_PARAMS 18817

/* 16 per-vertex features of the built index, bf16 bit patterns [n][16]:
 * log1p of indeg, outdeg, indeg*outdeg, indeg+outdeg, the sums over Pre(x)
 * of indeg and of outdeg, over Suc(x) of outdeg and of indeg (features 4-7 in
 * that order: Pre-indeg, Suc-outdeg, Pre-outdeg, Suc-indeg), popcounts of
 * DL_in, DL_out, BL_in, BL_out, popc(DL_in)*popc(DL_out), in-neighbours with
 * zero in-degree, out-neighbours with zero out-degree, and 1 for a landmark. */
dbl_status dbl_features(dbl_index *ix, uint16_t *feat, void *stream);

/* Coverage of sampled reachable pairs: count[c] = #{j : u[j] reaches c and c
 * reaches v[j]} over the pairs j kept (the pairs DL would decide if c were a
 * landmark, Lemma 1), by bit-parallel propagation, 256 pairs per pass.  A pair
 * is kept if reach[j] != 0 (reach may be NULL: all kept) and the index's first
 * base_slots landmark slots do not already decide it by the DL test; *kept
 * (may be NULL) receives their number.  target (may be NULL) receives
 * log1p(count[c]) / log1p(max count).  Synchronous. */
dbl_status dbl_coverage(dbl_index *ix, const int32_t *u, const int32_t *v, const uint8_t *reach, int64_t pairs,
                        int32_t base_slots, uint32_t *count, float *target, int64_t *kept, void *stream);

/* out[k]: the k vertices with the largest scores[n], ties by smaller id. */
dbl_status dbl_select_by_score(dbl_index *ix, const float *scores, int32_t k, int32_t *out, void *stream);
/* out[k]: greedy spread selection: the vertex of largest score (ties by
 * smaller id) among those not yet taken or excluded, then its in- and
 * out-neighbours are excluded, k times.  Vertices scored -inf or NaN are
 * never taken; slots left when no candidate remains get -1.  (A top-k of
 * landmarks tends to fall in one strongly connected component, where one of
 * them decides what all would; neighbours of a chosen vertex share its
 * component far more often than other vertices.) */
dbl_status dbl_select_spread(dbl_index *ix, const float *scores, int32_t k, int32_t *out, void *stream);
/* out[k]: the greedy selection of dbl_select_spread (spread != 0) or by score
 * alone (spread == 0; ties by smaller id, -1 for slots left empty), taking
 * no vertex of the strongly connected component of one of the index's first
 * covered_slots landmarks, i.e. no vertex whose DL_in and DL_out share one of
 * those landmarks' bits (Section 4.1's DL labels): every pair such a vertex
 * connects, that landmark connects too (u -> x -> landmark -> x -> v), so as a
 * landmark it would decide nothing more.  Applies insertion batches queued
 * under DBL_FLAG_DEFER first.  Synchronous. */
dbl_status dbl_select_uncovered(dbl_index *ix, const float *scores, int32_t k, int32_t covered_slots, int32_t spread,
                                int32_t *out, void *stream);

/* Network with initial parameters params_host[DBL_MLP_PARAMS] (host fp32).
 * Weights are kept in fp32 with bf16 copies for the tensor-core kernels. */
dbl_status dbl_mlp_create(const float *params_host, dbl_mlp **out, void *stream);
void dbl_mlp_destroy(dbl_mlp *m, void *stream);
/* Copy the current fp32 parameters to params_host[DBL_MLP_PARAMS]
 * (synchronises `stream`; reports errors as dbl_mlp_sync does). */
dbl_status dbl_mlp_params(dbl_mlp *m, float *params_host, void *stream);
/* y[r] = network(X[rows_idx ? rows_idx[r] : r]) for r < rows; X bf16 [.][16].
 * Runs on the tcgen05 tensor cores in 128-row tiles; without rows_idx and
 * with X 16-byte aligned the tiles arrive by TMA tensor copies (a tensor map
 * the driver refuses is DBL_ERR_CUDA).  The forward, gradient and training
 * calls are asynchronous; dbl_mlp_sync reports their errors. */
dbl_status dbl_mlp_forward(dbl_mlp *m, const uint16_t *X, const int32_t *rows_idx, int64_t rows, float *y,
                           void *stream);
/* Gradients (device fp32 [DBL_MLP_PARAMS]) and loss (device fp32, may be
 * NULL) of mean((y - target)^2)/2 over the rows, without changing the network. */
dbl_status dbl_mlp_gradients(dbl_mlp *m, const uint16_t *X, const float *target, const int32_t *rows_idx,
                             int64_t rows, float *grads, float *loss, void *stream);
/* One SGD-with-momentum step on the rows: v = momentum*v + grad; p -= lr*v. */
dbl_status dbl_mlp_train_step(dbl_mlp *m, const uint16_t *X, const float *target, const int32_t *rows_idx,
                              int64_t rows, float lr, float momentum, float *loss, void *stream);
/* Wait for `stream`; DBL_ERR_TIMEOUT if a tensor-core kernel of this network
 * gave up a bounded wait since it was created (its outputs are invalid). */
dbl_status dbl_mlp_sync(dbl_mlp *m, void *stream);
const char *dbl_mlp_last_error(const dbl_mlp *m);

/* Write the index to the file at `path` (created or truncated): its base
 * graph, landmark and leaf choices, labels (Definitions 1-2), per-vertex
 * adjacency metadata and the used part of the inserted-edge pools, the vertex
 * count and the stored-edge count; insertion batches queued under
 * DBL_FLAG_DEFER are applied first.  Snapshots are not written.  The file's
 * size is about the device memory the index uses minus its frontier and
 * scratch buffers.  Writes through a 64 MB pinned host buffer.  Synchronous.
 * DBL_ERR_IO if the file cannot be written (the index is unchanged either
 * way); DBL_ERR_POISONED for a poisoned index. */
dbl_status dbl_save(dbl_index *ix, const char *path, void *stream);

/* Read an index written by dbl_save into a new index on the current device.
 * `opt` (NULL: defaults) supplies the allocator, flags, team and query
 * options; the capacities (edge_capacity, vertex_capacity, initial_slots)
 * are the saved index's.  The loaded index answers every query and takes
 * every later insertion exactly as the saved one would.  While the call
 * runs, the base graph and the landmark and leaf arrays pass through
 * temporary device buffers taken with cudaMalloc (about 4 bytes per edge and
 * 9 per vertex; not from the allocator in opt) and a 64 MB pinned host buffer.
 * Synchronous.  DBL_ERR_IO if the file is missing, short, of another format
 * version or inconsistent; DBL_ERR_OOM as dbl_build. */
dbl_status dbl_load(const char *path, const dbl_options *opt, void *stream, dbl_index **out);

/* Message of the last error on this index (or of the last failed build when
 * ix is NULL).  Valid until the next call on the index. */
const char *dbl_last_error(const dbl_index *ix);

/* Free the index and all its device memory (stream-ordered on `stream`). */
void dbl_destroy(dbl_index *ix, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DBL_H */
