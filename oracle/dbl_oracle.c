/*
 * CPU oracle for the DBL reachability index (arXiv 2101.09441).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential
 * statement of what the index computes, used to check the CUDA library
 * element by element.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header or table with the
 * CUDA library, and the library never calls it.
 *
 * What it follows, step by step:
 *   - Landmark choice: rank by M(u) = |Pre(u)| * |Suc(u)|, keep the top k
 *     (Section 4.1, landmark heuristic); ties by smaller vertex id.  The other
 *     rankings of Table 3 (Section 6, "Label Node Selection"): A = max(|Pre|,
 *     |Suc|), B = min(|Pre|, |Suc|), C = |Pre| + |Suc|.
 *   - Leaves: zero in-degree vertices seed BL_in, zero out-degree vertices seed
 *     BL_out (Definition 2, "BL label"); bucket h(v) by Fibonacci hashing
 *     (Knuth, TAOCP vol. 3, 6.4), since the paper leaves h open.  Section 6
 *     ("Label Node Selection") widens the leaf set to every u with M(u) <= r;
 *     a leaf with M(u) > 0 has both neighbour kinds and here seeds both BL_in
 *     and BL_out (the paper does not say; Lemma 2 holds for any leaf sets).
 *   - Build: one queue BFS per landmark forward (DL_in) and backward (DL_out),
 *     and one multi-source BFS per leaf bucket (Algorithm 1 and the paragraph
 *     after it).  A landmark / leaf labels itself (as Figure 1 shows), and
 *     "bit already set" is the visited test.
 *   - Insertion of (u, v): skip when DL_out(u) and DL_in(v) intersect
 *     (Algorithm 3, first test); otherwise a pruned BFS from v over Suc that
 *     ORs DL_in(u) into every x until DL_in(u) is contained in DL_in(x), v
 *     itself tested first (as the text and Figure 2 do); the DL_out mirror
 *     runs from u over Pre with DL_out(v) (Section 5); BL_in / BL_out the same
 *     way on their own words.
 *   - Vertex insertion (Section 1: insert-only graphs gain edges and
 *     vertices): new vertices are isolated, so their labels are empty; they
 *     join neither the landmarks nor the leaves (both sets are fixed at build).
 *   - Query (Algorithm 2): u == v answers true (Des/Anc include the vertex,
 *     Table 1); then DL intersection -> true; BL containment fails -> false;
 *     Theorem 1 -> false; Theorem 2 -> false; else a BFS from u with a visited
 *     set that tests x == v, then the DL prune, then the BL prune.
 *
 * Label layout: label arrays are [n][words] uint64, landmark slot i at word
 * i/64 bit i%64, bucket b at word b/64 bit b%64.  A landmark slot holding -1
 * is empty.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
    ORC_UNDECIDED = 0,
    ORC_SELF = 1,
    ORC_DL = 2,
    ORC_BL = 3,
    ORC_THM1 = 4,
    ORC_THM2 = 5,
    ORC_BFS_POS = 6,
    ORC_BFS_NEG = 7
};

typedef struct {
    int32_t len, cap;
    int32_t *v;
} adjlist;

typedef struct {
    int32_t n, k, kp, wd, wb;
    adjlist *suc, *pre;
    uint64_t *dl_in, *dl_out, *bl_in, *bl_out;
    int32_t *landmarks;
    int32_t *leaf_bucket;
    uint8_t *leaf_role;
    int32_t *queue; /* sequential scratch, n entries */
    uint64_t ins_skipped, ins_applied, ins_visits;
} orc_index;

static int adj_push(adjlist *a, int32_t x)
{
    if (a->len == a->cap) {
        int32_t nc = a->cap ? a->cap * 2 : 4;
        int32_t *nv = (int32_t *)realloc(a->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return 0;
        a->v = nv;
        a->cap = nc;
    }
    a->v[a->len++] = x;
    return 1;
}

void orc_destroy(orc_index *h)
{
    if (!h) return;
    if (h->suc)
        for (int32_t i = 0; i < h->n; ++i) free(h->suc[i].v);
    if (h->pre)
        for (int32_t i = 0; i < h->n; ++i) free(h->pre[i].v);
    free(h->suc);
    free(h->pre);
    free(h->dl_in);
    free(h->dl_out);
    free(h->bl_in);
    free(h->bl_out);
    free(h->landmarks);
    free(h->leaf_bucket);
    free(h->leaf_role);
    free(h->queue);
    free(h);
}

/* G from a CSR (any row order); k landmark slots, kp leaf buckets. */
orc_index *orc_create(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t k, int32_t kp)
{
    if (n < 0 || k < 1 || kp < 1) return NULL;
    orc_index *h = (orc_index *)calloc(1, sizeof(orc_index));
    if (!h) return NULL;
    h->n = n;
    h->k = k;
    h->kp = kp;
    h->wd = (k + 63) / 64;
    h->wb = (kp + 63) / 64;
    size_t nn = n > 0 ? (size_t)n : 1;
    h->suc = (adjlist *)calloc(nn, sizeof(adjlist));
    h->pre = (adjlist *)calloc(nn, sizeof(adjlist));
    h->dl_in = (uint64_t *)calloc(nn * h->wd, 8);
    h->dl_out = (uint64_t *)calloc(nn * h->wd, 8);
    h->bl_in = (uint64_t *)calloc(nn * h->wb, 8);
    h->bl_out = (uint64_t *)calloc(nn * h->wb, 8);
    h->landmarks = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    h->leaf_bucket = (int32_t *)malloc(sizeof(int32_t) * nn);
    h->leaf_role = (uint8_t *)calloc(nn, 1);
    h->queue = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!h->suc || !h->pre || !h->dl_in || !h->dl_out || !h->bl_in || !h->bl_out || !h->landmarks ||
        !h->leaf_bucket || !h->leaf_role || !h->queue) {
        orc_destroy(h);
        return NULL;
    }
    for (int32_t i = 0; i < k; ++i) h->landmarks[i] = -1;
    for (int32_t v = 0; v < n; ++v) h->leaf_bucket[v] = -1;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (v < 0 || v >= n || !adj_push(&h->suc[u], v) || !adj_push(&h->pre[v], u)) {
                orc_destroy(h);
                return NULL;
            }
        }
    return h;
}

/* ---------------------------------------------------------------- labels */

static inline int bit_get(const uint64_t *w, int32_t i) { return (int)((w[i >> 6] >> (i & 63)) & 1u); }

/* DL_Intersec(x, y): DL_out(x) and DL_in(y) share a landmark (Algorithm 2). */
static int dl_intersec(const orc_index *h, int32_t x, int32_t y)
{
    const uint64_t *a = h->dl_out + (size_t)x * h->wd, *b = h->dl_in + (size_t)y * h->wd;
    for (int32_t w = 0; w < h->wd; ++w)
        if (a[w] & b[w]) return 1;
    return 0;
}

/* BL_Contain(x, y): BL_in(x) within BL_in(y) and BL_out(y) within BL_out(x) (Algorithm 2). */
static int bl_contain(const orc_index *h, int32_t x, int32_t y)
{
    const uint64_t *ix = h->bl_in + (size_t)x * h->wb, *iy = h->bl_in + (size_t)y * h->wb;
    const uint64_t *ox = h->bl_out + (size_t)x * h->wb, *oy = h->bl_out + (size_t)y * h->wb;
    for (int32_t w = 0; w < h->wb; ++w) {
        if (ix[w] & ~iy[w]) return 0;
        if (oy[w] & ~ox[w]) return 0;
    }
    return 1;
}

/* Landmarks: top-k by M(u) = |Pre(u)|*|Suc(u)| (Section 4.1), ties by id. */
static const int64_t *g_rank_M;
static int cmp_rank(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_rank_M[a] != g_rank_M[b]) return g_rank_M[a] > g_rank_M[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* Ranking key of v: rule 0 = |Pre| * |Suc| (the paper's), 1 = A = max,
 * 2 = B = min, 3 = C = sum of |Pre| and |Suc| (Table 3). */
static int64_t rank_key(const orc_index *h, int32_t v, int rule)
{
    const int64_t p = h->pre[v].len, s = h->suc[v].len;
    switch (rule) {
    case 1: return p > s ? p : s;
    case 2: return p < s ? p : s;
    case 3: return p + s;
    default: return p * s;
    }
}

int orc_rank_landmarks(const orc_index *h, int rule, int32_t *out)
{
    int32_t n = h->n;
    if (rule < 0 || rule > 3) return 1;
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!M || !ids) { free(M); free(ids); return 2; }
    for (int32_t v = 0; v < n; ++v) {
        M[v] = rank_key(h, v, rule);
        ids[v] = v;
    }
    g_rank_M = M;
    qsort(ids, (size_t)n, sizeof(int32_t), cmp_rank);
    for (int32_t i = 0; i < h->k; ++i) out[i] = i < n ? ids[i] : -1;
    free(M);
    free(ids);
    return 0;
}

/* Bucket of leaf v among kp buckets: floor(frac(v * phi) * kp) with phi the
 * 64-bit golden ratio; for kp = 2^b this is Fibonacci hashing v*phi >> (64-b). */
static int32_t leaf_hash(int32_t v, int32_t kp)
{
    uint64_t x = (uint64_t)(uint32_t)v * 0x9E3779B97F4A7C15ULL;
    return (int32_t)(((unsigned __int128)x * (uint64_t)kp) >> 64);
}

int32_t orc_leaf_hash(int32_t v, int32_t kp) { return leaf_hash(v, kp); }

int orc_degree_landmarks(const orc_index *h, int32_t *out) { return orc_rank_landmarks(h, 0, out); }

/* Leaves by threshold (Section 6, "Label Node Selection"): v is a leaf iff
 * M(v) = |Pre(v)| * |Suc(v)| <= r.  With M(v) = 0 its roles are those of
 * Definition 2 (zero in-degree seeds BL_in, zero out-degree seeds BL_out);
 * a leaf with M(v) > 0 seeds both.  r = 0 is orc_zero_degree_leaves. */
int orc_threshold_leaves(const orc_index *h, int64_t r, int32_t *bucket, uint8_t *role)
{
    if (r < 0) return 1;
    for (int32_t v = 0; v < h->n; ++v) {
        const int64_t M = (int64_t)h->pre[v].len * (int64_t)h->suc[v].len;
        uint8_t ro = 0;
        if (M == 0) ro = (uint8_t)((h->pre[v].len == 0 ? 1 : 0) | (h->suc[v].len == 0 ? 2 : 0));
        else if (M <= r) ro = 3;
        role[v] = ro;
        bucket[v] = ro ? leaf_hash(v, h->kp) : -1;
    }
    return 0;
}

/* Leaves: zero in-degree -> role bit 0 (seeds BL_in), zero out-degree -> role
 * bit 1 (seeds BL_out) (Definition 2). */
int orc_zero_degree_leaves(const orc_index *h, int32_t *bucket, uint8_t *role)
{
    for (int32_t v = 0; v < h->n; ++v) {
        uint8_t r = (uint8_t)((h->pre[v].len == 0 ? 1 : 0) | (h->suc[v].len == 0 ? 2 : 0));
        role[v] = r;
        bucket[v] = r ? leaf_hash(v, h->kp) : -1;
    }
    return 0;
}

/* Algorithm 1 for one bit: BFS over `adj` from the seed list, setting `bit` in
 * lab[x] for every vertex reached; a set bit is the visited test. */
static void bfs_set_bit(int32_t n, const adjlist *adj, uint64_t *lab, int32_t words, int32_t bit,
                        const int32_t *seeds, int32_t nseeds, int32_t *queue)
{
    const uint64_t mask = 1ULL << (bit & 63);
    const int32_t wi = bit >> 6;
    int64_t head = 0, tail = 0;
    for (int32_t s = 0; s < nseeds; ++s) {
        uint64_t *w = lab + (size_t)seeds[s] * words + wi;
        if (!(__atomic_load_n(w, __ATOMIC_RELAXED) & mask)) {
            __atomic_fetch_or(w, mask, __ATOMIC_RELAXED);
            queue[tail++] = seeds[s];
        }
    }
    while (head < tail) {
        int32_t p = queue[head++];
        for (int32_t e = 0; e < adj[p].len; ++e) {
            int32_t x = adj[p].v[e];
            uint64_t *w = lab + (size_t)x * words + wi;
            if (__atomic_load_n(w, __ATOMIC_RELAXED) & mask) continue;
            __atomic_fetch_or(w, mask, __ATOMIC_RELAXED);
            queue[tail++] = x;
        }
    }
    (void)n;
}

/*
 * Build all four labels (Algorithm 1): landmarks[k] (-1 = empty slot),
 * leaf_bucket[n] (-1 = not a leaf), leaf_role[n] (bit0 BL_in seed, bit1 BL_out
 * seed).  nthreads > 1 runs the independent per-bit BFSs in parallel (the
 * multi-core form); the result does not depend on it.
 */
int orc_build(orc_index *h, const int32_t *landmarks, const int32_t *leaf_bucket,
              const uint8_t *leaf_role, int nthreads)
{
    int32_t n = h->n, k = h->k, kp = h->kp;
    for (int32_t i = 0; i < k; ++i) {
        if (landmarks[i] >= n) return 1;
        h->landmarks[i] = landmarks[i] < 0 ? -1 : landmarks[i];
    }
    for (int32_t v = 0; v < n; ++v) {
        if (leaf_bucket[v] >= kp) return 1;
        h->leaf_bucket[v] = leaf_bucket[v];
        h->leaf_role[v] = leaf_bucket[v] < 0 ? 0 : (uint8_t)(leaf_role[v] & 3);
    }
    size_t nn = n > 0 ? (size_t)n : 1;
    memset(h->dl_in, 0, nn * h->wd * 8);
    memset(h->dl_out, 0, nn * h->wd * 8);
    memset(h->bl_in, 0, nn * h->wb * 8);
    memset(h->bl_out, 0, nn * h->wb * 8);

    /* seed lists per bucket and direction */
    int32_t *cnt = (int32_t *)calloc((size_t)kp * 2 + 1, sizeof(int32_t));
    int32_t *off = (int32_t *)calloc((size_t)kp * 2 + 1, sizeof(int32_t));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * nn * 2);
    if (!cnt || !off || !list) { free(cnt); free(off); free(list); return 2; }
    for (int32_t v = 0; v < n; ++v) {
        if (h->leaf_role[v] & 1) cnt[h->leaf_bucket[v]]++;
        if (h->leaf_role[v] & 2) cnt[kp + h->leaf_bucket[v]]++;
    }
    for (int32_t i = 0; i < 2 * kp; ++i) off[i + 1] = off[i] + cnt[i];
    memcpy(cnt, off, sizeof(int32_t) * (size_t)(2 * kp));
    for (int32_t v = 0; v < n; ++v) {
        if (h->leaf_role[v] & 1) list[cnt[h->leaf_bucket[v]]++] = v;
        if (h->leaf_role[v] & 2) list[cnt[kp + h->leaf_bucket[v]]++] = v;
    }

    /* jobs: 2k landmark BFSs (fwd, bwd) then 2kp bucket BFSs */
    int64_t njobs = 2 * (int64_t)k + 2 * (int64_t)kp;
    if (nthreads < 1) nthreads = 1;
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        int32_t *q = (int32_t *)malloc(sizeof(int32_t) * nn);
        if (!q) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < njobs; ++j) {
            if (!q) continue;
            if (j < 2 * k) {
                int32_t i = (int32_t)(j >> 1);
                int32_t l = h->landmarks[i];
                if (l < 0) continue;
                if ((j & 1) == 0) bfs_set_bit(n, h->suc, h->dl_in, h->wd, i, &l, 1, q);
                else bfs_set_bit(n, h->pre, h->dl_out, h->wd, i, &l, 1, q);
            } else {
                int64_t jj = j - 2 * k;
                int32_t b = (int32_t)(jj >> 1);
                if ((jj & 1) == 0)
                    bfs_set_bit(n, h->suc, h->bl_in, h->wb, b, list + off[b], off[b + 1] - off[b], q);
                else
                    bfs_set_bit(n, h->pre, h->bl_out, h->wb, b, list + off[kp + b],
                                off[kp + b + 1] - off[kp + b], q);
            }
        }
        free(q);
    }
    free(cnt);
    free(off);
    free(list);
    return failed ? 2 : 0;
}

/* ------------------------------------------------------------- insertion */

/* Pruned BFS of Algorithm 3 on one label kind: OR S into every vertex reached
 * from `start` over `adj` whose label does not already contain S; a vertex
 * that already contains S is pruned with all it would lead to.  The start
 * vertex itself is tested and updated first. */
static uint64_t pruned_or(orc_index *h, const adjlist *adj, uint64_t *lab, int32_t words,
                          const uint64_t *S, int32_t start)
{
    uint64_t visits = 0;
    int64_t head = 0, tail = 0;
#define CONTAINED(x)                                                                   \
    ({                                                                                 \
        const uint64_t *L_ = lab + (size_t)(x) * words;                                \
        int c_ = 1;                                                                    \
        for (int32_t w_ = 0; w_ < words; ++w_)                                         \
            if (S[w_] & ~L_[w_]) { c_ = 0; break; }                                    \
        c_;                                                                            \
    })
#define OR_IN(x)                                                                       \
    do {                                                                               \
        uint64_t *L_ = lab + (size_t)(x) * words;                                      \
        for (int32_t w_ = 0; w_ < words; ++w_) L_[w_] |= S[w_];                        \
    } while (0)
    ++visits;
    if (CONTAINED(start)) return visits;
    OR_IN(start);
    h->queue[tail++] = start;
    while (head < tail) {
        int32_t p = h->queue[head++];
        for (int32_t e = 0; e < adj[p].len; ++e) {
            int32_t x = adj[p].v[e];
            ++visits;
            if (!CONTAINED(x)) {
                OR_IN(x);
                h->queue[tail++] = x;
            }
        }
    }
#undef CONTAINED
#undef OR_IN
    return visits;
}

/*
 * Insert edge (u, v) and repair all four labels (Algorithm 3 and its mirrors).
 * Self-loops change nothing and are not stored.  Returns 0, 1 on an invalid
 * id, 2 on allocation failure.
 */
int orc_insert_edge(orc_index *h, int32_t u, int32_t v)
{
    if (u < 0 || v < 0 || u >= h->n || v >= h->n) return 1;
    if (u == v) return 0;
    int skip = dl_intersec(h, u, v);
    if (!adj_push(&h->suc[u], v) || !adj_push(&h->pre[v], u)) return 2;
    if (skip) {
        h->ins_skipped++;
        return 0;
    }
    h->ins_applied++;
    uint64_t S[64];
    int32_t wmax = h->wd > h->wb ? h->wd : h->wb;
    if (wmax > 64) return 1;
    /* DL_in: add DL_in(u) to Des(v) */
    memcpy(S, h->dl_in + (size_t)u * h->wd, 8 * (size_t)h->wd);
    h->ins_visits += pruned_or(h, h->suc, h->dl_in, h->wd, S, v);
    /* DL_out (mirror): add DL_out(v) to Anc(u) */
    memcpy(S, h->dl_out + (size_t)v * h->wd, 8 * (size_t)h->wd);
    h->ins_visits += pruned_or(h, h->pre, h->dl_out, h->wd, S, u);
    /* BL_in: add BL_in(u) to Des(v) */
    memcpy(S, h->bl_in + (size_t)u * h->wb, 8 * (size_t)h->wb);
    h->ins_visits += pruned_or(h, h->suc, h->bl_in, h->wb, S, v);
    /* BL_out: add BL_out(v) to Anc(u) */
    memcpy(S, h->bl_out + (size_t)v * h->wb, 8 * (size_t)h->wb);
    h->ins_visits += pruned_or(h, h->pre, h->bl_out, h->wb, S, u);
    return 0;
}

int orc_insert_edges(orc_index *h, const int32_t *src, const int32_t *dst, int64_t b)
{
    for (int64_t i = 0; i < b; ++i) {
        int rc = orc_insert_edge(h, src[i], dst[i]);
        if (rc) return rc;
    }
    return 0;
}

/* ----------------------------------------------------------------- query */

/* Algorithm 2 for one pair; stamp/queue are caller scratch (n entries each),
 * epoch a fresh stamp value.  Writes the deciding rule to *code. */
static int query_one(const orc_index *h, int32_t u, int32_t v, uint8_t *code, int32_t *stamp,
                     int32_t epoch, int32_t *queue, uint64_t *expanded, uint64_t *scanned)
{
    if (u == v) { *code = ORC_SELF; return 1; }
    if (dl_intersec(h, u, v)) { *code = ORC_DL; return 1; }
    if (!bl_contain(h, u, v)) { *code = ORC_BL; return 0; }
    if (dl_intersec(h, v, u)) { *code = ORC_THM1; return 0; }
    if (dl_intersec(h, u, u) || dl_intersec(h, v, v)) { *code = ORC_THM2; return 0; }
    int64_t head = 0, tail = 0;
    stamp[u] = epoch;
    queue[tail++] = u;
    while (head < tail) {
        int32_t w = queue[head++];
        ++*expanded;
        const adjlist *a = &h->suc[w];
        for (int32_t e = 0; e < a->len; ++e) {
            int32_t x = a->v[e];
            ++*scanned;
            if (x == v) { *code = ORC_BFS_POS; return 1; }
            if (dl_intersec(h, u, x)) continue;
            if (!bl_contain(h, x, v)) continue;
            if (stamp[x] == epoch) continue;
            stamp[x] = epoch;
            queue[tail++] = x;
        }
    }
    *code = ORC_BFS_NEG;
    return 0;
}

/* Batch of q queries; ans/code per pair; stats[0..7] counts per code,
 * stats[8] BFS vertices expanded, stats[9] BFS edges scanned.  Returns 0 or 1
 * on an invalid id (nothing written past it is meaningful). */
int orc_query(const orc_index *h, const int32_t *qu, const int32_t *qv, int64_t q, uint8_t *ans,
              uint8_t *code, uint64_t *stats, int nthreads)
{
    int32_t n = h->n;
    for (int64_t i = 0; i < q; ++i)
        if (qu[i] < 0 || qu[i] >= n || qv[i] < 0 || qv[i] >= n) return 1;
    if (nthreads < 1) nthreads = 1;
    uint64_t st[10] = {0};
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        size_t nn = n > 0 ? (size_t)n : 1;
        int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * nn);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * nn);
        uint64_t loc[10] = {0};
        if (!stamp || !queue) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int32_t i = 0; i < n; ++i) stamp[i] = 0;
        }
        int32_t epoch = 0;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < q; ++i) {
            if (!stamp || !queue) continue;
            uint8_t c = 0;
            ++epoch;
            if (epoch == 0x7fffffff) {
                for (int32_t j = 0; j < n; ++j) stamp[j] = 0;
                epoch = 1;
            }
            ans[i] = (uint8_t)query_one(h, qu[i], qv[i], &c, stamp, epoch, queue, &loc[8], &loc[9]);
            if (code) code[i] = c;
            loc[c]++;
        }
        for (int j = 0; j < 10; ++j) {
#pragma omp atomic
            st[j] += loc[j];
        }
        free(stamp);
        free(queue);
    }
    if (stats) memcpy(stats, st, sizeof(st));
    return failed ? 2 : 0;
}

/* ------------------------------------------------------------- accessors */

int32_t orc_n(const orc_index *h) { return h->n; }
int32_t orc_words_dl(const orc_index *h) { return h->wd; }
int32_t orc_words_bl(const orc_index *h) { return h->wb; }

void orc_labels(const orc_index *h, uint64_t *dl_in, uint64_t *dl_out, uint64_t *bl_in, uint64_t *bl_out)
{
    size_t nn = (size_t)h->n;
    if (dl_in) memcpy(dl_in, h->dl_in, nn * h->wd * 8);
    if (dl_out) memcpy(dl_out, h->dl_out, nn * h->wd * 8);
    if (bl_in) memcpy(bl_in, h->bl_in, nn * h->wb * 8);
    if (bl_out) memcpy(bl_out, h->bl_out, nn * h->wb * 8);
}

/* Current adjacency as CSR-out (row order = insertion order). */
int64_t orc_num_edges(const orc_index *h)
{
    int64_t m = 0;
    for (int32_t v = 0; v < h->n; ++v) m += h->suc[v].len;
    return m;
}

void orc_csr(const orc_index *h, int64_t *row_ptr, int32_t *col)
{
    int64_t e = 0;
    row_ptr[0] = 0;
    for (int32_t v = 0; v < h->n; ++v) {
        for (int32_t j = 0; j < h->suc[v].len; ++j) col[e++] = h->suc[v].v[j];
        row_ptr[v + 1] = e;
    }
}

/* Vertex insertion: count isolated vertices n .. n + count - 1, with empty
 * labels and no edges, not landmarks and not leaves.  Returns 0, 1 (count
 * negative or the ids would not fit in int32) or 2 (out of memory; the index
 * is then unusable). */
int orc_add_vertices(orc_index *h, int32_t count)
{
    if (count < 0 || (int64_t)h->n + count >= ((int64_t)1 << 31)) return 1;
    if (count == 0) return 0;
    const size_t n0 = (size_t)h->n, n1 = n0 + (size_t)count;
    adjlist *su = (adjlist *)realloc(h->suc, sizeof(adjlist) * n1);
    if (!su) return 2;
    h->suc = su;
    adjlist *pr = (adjlist *)realloc(h->pre, sizeof(adjlist) * n1);
    if (!pr) return 2;
    h->pre = pr;
    memset(h->suc + n0, 0, sizeof(adjlist) * (size_t)count);
    memset(h->pre + n0, 0, sizeof(adjlist) * (size_t)count);
    uint64_t **lab[4] = {&h->dl_in, &h->dl_out, &h->bl_in, &h->bl_out};
    const int32_t words[4] = {h->wd, h->wd, h->wb, h->wb};
    for (int i = 0; i < 4; ++i) {
        uint64_t *t = (uint64_t *)realloc(*lab[i], 8 * n1 * (size_t)words[i]);
        if (!t) return 2;
        memset(t + n0 * (size_t)words[i], 0, 8 * (size_t)count * (size_t)words[i]);
        *lab[i] = t;
    }
    int32_t *lb = (int32_t *)realloc(h->leaf_bucket, sizeof(int32_t) * n1);
    if (!lb) return 2;
    h->leaf_bucket = lb;
    uint8_t *lr = (uint8_t *)realloc(h->leaf_role, n1);
    if (!lr) return 2;
    h->leaf_role = lr;
    int32_t *q = (int32_t *)realloc(h->queue, sizeof(int32_t) * n1);
    if (!q) return 2;
    h->queue = q;
    for (size_t v = n0; v < n1; ++v) {
        h->leaf_bucket[v] = -1;
        h->leaf_role[v] = 0;
    }
    h->n = (int32_t)n1;
    return 0;
}

/* Save the labels and adjacency lengths; orc_rewind returns to them (so a
 * timed step can be repeated from the same state); not across a vertex
 * insertion.  Returns 0 or 2. */
static uint64_t *g_mark_lab[4];
static int32_t *g_mark_len[2];
static const orc_index *g_mark_owner;
static int32_t g_mark_n;

int orc_mark(orc_index *h)
{
    size_t nn = h->n > 0 ? (size_t)h->n : 1;
    size_t sz[4] = {nn * h->wd, nn * h->wd, nn * h->wb, nn * h->wb};
    uint64_t *src[4] = {h->dl_in, h->dl_out, h->bl_in, h->bl_out};
    for (int i = 0; i < 4; ++i) {
        free(g_mark_lab[i]);
        g_mark_lab[i] = (uint64_t *)malloc(8 * sz[i]);
        if (!g_mark_lab[i]) return 2;
        memcpy(g_mark_lab[i], src[i], 8 * sz[i]);
    }
    for (int d = 0; d < 2; ++d) {
        free(g_mark_len[d]);
        g_mark_len[d] = (int32_t *)malloc(sizeof(int32_t) * nn);
        if (!g_mark_len[d]) return 2;
        for (int32_t v = 0; v < h->n; ++v) g_mark_len[d][v] = d ? h->pre[v].len : h->suc[v].len;
    }
    g_mark_owner = h;
    g_mark_n = h->n;
    return 0;
}

int orc_rewind(orc_index *h)
{
    if (g_mark_owner != h || g_mark_n != h->n) return 1;
    size_t nn = h->n > 0 ? (size_t)h->n : 1;
    size_t sz[4] = {nn * h->wd, nn * h->wd, nn * h->wb, nn * h->wb};
    uint64_t *dst[4] = {h->dl_in, h->dl_out, h->bl_in, h->bl_out};
    for (int i = 0; i < 4; ++i) memcpy(dst[i], g_mark_lab[i], 8 * sz[i]);
    for (int32_t v = 0; v < h->n; ++v) {
        h->suc[v].len = g_mark_len[0][v];
        h->pre[v].len = g_mark_len[1][v];
    }
    return 0;
}

void orc_insert_stats(const orc_index *h, uint64_t *out3)
{
    out3[0] = h->ins_skipped;
    out3[1] = h->ins_applied;
    out3[2] = h->ins_visits;
}
