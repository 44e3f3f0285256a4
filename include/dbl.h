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
 *               (Definition 2 and the hashing paragraph, Section 4.1).
 * Reachability is reflexive: Des(u) and Anc(u) contain u (Table 1).
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers unless the name ends in _host.
 *     They are borrowed: the caller keeps them alive until the stream has
 *     passed the call.  Calls are ordered on `stream` (a cudaStream_t; NULL
 *     means the legacy default stream).
 *   - Vertex ids are int32 in [0, n).  Labels are uint64 words: landmark slot
 *     i is word i/64 bit i%64, bucket b is word b/64 bit b%64.
 *   - An invalid argument is reported as DBL_ERR_INVALID before any state
 *     changes.  Running out of the index's edge capacity is DBL_ERR_CAPACITY,
 *     with the index unchanged.  A device loop that exceeds its iteration
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
    DBL_ERR_POISONED = 7  /* an earlier timeout poisoned the index */
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
    DBL_FLAG_TIMING = 4      /* bracket kernels with CUDA events (dbl_timings) */
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
                              0: max(2^20, m/4) */
    int32_t flags;         /* DBL_FLAG_* */
    int32_t bfs_words;     /* 64-query words per search wave (1..64); 0: 16 */
    int32_t team;          /* lanes per expansion task (4, 8, 16, 32); 0: 8 */
    int32_t reserved[7];
} dbl_options;

/* Fill *opt with the defaults above. */
void dbl_default_options(dbl_options *opt);

/*
 * Build the index for G (Algorithm 1 and the BL construction of Section 4.1).
 *   landmarks[k]   landmark of slot i, or -1 for an empty slot; NULL: the
 *                  top-k vertices by M(u) = |Pre(u)| * |Suc(u)| (Section 4.1,
 *                  landmark heuristic), ties by smaller id.
 *   k              multiple of 64, 64..256.
 *   leaf_buckets[n] bucket in [0, kprime) of a leaf, -1 for a non-leaf;
 *                  NULL: zero in-degree vertices seed BL_in and zero
 *                  out-degree vertices seed BL_out (Definition 2), bucket
 *                  h(v) = floor(frac(v * 0x9E3779B97F4A7C15 / 2^64) * kprime)
 *                  (Fibonacci hashing; the paper leaves h open).
 *   leaf_roles[n]  bit0: seeds BL_in, bit1: seeds BL_out; required when
 *                  leaf_buckets is given, ignored otherwise.
 *   kprime         multiple of 64, 64..256.
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
 *     before any stream capture;
 *   - all calls in the process share the one array: calls whose device work
 *     overlaps (on different streams, or on different indexes of the same
 *     device) race on it and must be ordered by the caller.  Each call writes
 *     every scratch entry it reads, so nothing left by an earlier call is used.
 */
dbl_status dbl_insert_edges_noalloc(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b,
                                    void *stream);

/* Host-buffer forms: copy inputs from host memory (pinned or pageable) to
 * the device, run the call, and copy results back, in overlapped chunks
 * (the transfer overlap of Section 6.6).  Synchronous. */
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

/* Save / restore labels and inserted adjacency in snapshot slot 0..3
 * (device-to-device copies on `stream`).  dbl_restore clears a poisoned index. */
dbl_status dbl_snapshot(dbl_index *ix, int slot, void *stream);
dbl_status dbl_restore(dbl_index *ix, int slot, void *stream);

/* Wait for `stream` and return the first error latched on the device. */
dbl_status dbl_sync(dbl_index *ix, void *stream);

/*
 * Counters since build (synchronises `stream`):
 *  [0..7]  queries decided per DBL_CODE_*     [8]  frontier levels run
 *  [9]     expansion tasks                    [10] edges relaxed
 *  [11]    inserted edges applied             [12] insertions skipped (u reached v)
 *  [13]    self-loops ignored                 [14] search waves
 *  [15]    inserted edges stored
 */
dbl_status dbl_stats(dbl_index *ix, uint64_t counters[16], void *stream);

/* With DBL_FLAG_TIMING: device time (ms, from CUDA events recorded on the
 * launching stream) and launch count per DBL_KERNEL_* class since the last
 * call; synchronises `stream`.  Without the flag both arrays are zero. */
dbl_status dbl_timings(dbl_index *ix, double ms[8], uint64_t launches[8], void *stream);

/* Facts about the index: [0] n, [1] k, [2] kprime, [3] inserted edges stored,
 * [4] edge capacity, [5] base edges m, [6] label record bytes per vertex,
 * [7] option flags, [8] kernels launched so far, [9] words per record half;
 * [10..15] zero. */
dbl_status dbl_info(const dbl_index *ix, int64_t info[16]);

/* Message of the last error on this index (or of the last failed build when
 * ix is NULL).  Valid until the next call on the index. */
const char *dbl_last_error(const dbl_index *ix);

/* Free the index and all its device memory (stream-ordered on `stream`). */
void dbl_destroy(dbl_index *ix, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DBL_H */
