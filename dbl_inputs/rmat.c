/*
 * Seeded synthetic inputs for the DBL reachability index: R-MAT graphs, edge
 * insertion streams and mixed query streams.
 *
 * This module holds no part of the index's arithmetic (no labels, no label
 * tests, no propagation).  It is shared by the CPU oracle, the tests and the
 * benchmark so that both sides of every parity check see the same inputs.
 *
 * Randomness: every draw is the i-th output of a splitmix64 generator
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) whose state starts at a per-purpose key derived from the seed.
 * Draws are addressed by counter, so the output does not depend on the number
 * of threads.
 *
 * R-MAT: Chakrabarti, Zhan and Faloutsos, "R-MAT: a recursive model for graph
 * mining", SDM 2004.  Quadrant probabilities (a, b, c, d=1-a-b-c); quadrant b
 * sets the destination bit, quadrant c the source bit.  No noise.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i = 0, 1, ...) of splitmix64 started from state `key`. */
static inline uint64_t sm64_at(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

/* Independent stream per purpose. */
enum { TAG_PERM = 1, TAG_EDGES = 2, TAG_INSERT = 3, TAG_QUERY = 4, TAG_SIZES = 5 };
static inline uint64_t stream_key(uint64_t seed, uint64_t tag)
{
    return mix64(seed ^ (tag * 0xD1B54A32D192ED03ULL));
}

/* uniform integer in [0, bound) by multiply-shift (Lemire 2019). */
static inline uint64_t bounded(uint64_t r, uint64_t bound)
{
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

static inline double unit53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

uint64_t dblgen_splitmix64_at(uint64_t key, uint64_t i) { return sm64_at(key, i); }
uint64_t dblgen_stream_key(uint64_t seed, uint64_t tag) { return stream_key(seed, tag); }

/* Fisher-Yates permutation of [0, n) keyed by seed. */
static void make_perm(int32_t n, uint64_t seed, int32_t *perm)
{
    uint64_t key = stream_key(seed, TAG_PERM);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = (int64_t)n - 1; i > 0; --i) {
        int64_t j = (int64_t)bounded(sm64_at(key, (uint64_t)(n - 1 - i)), (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

int dblgen_permutation(int32_t n, uint64_t seed, int32_t *perm)
{
    if (n < 0 || !perm) return 1;
    make_perm(n, seed, perm);
    return 0;
}

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* k-th smallest (0-based) of v[0..len); reorders v. */
static int64_t select_kth(int64_t *v, int64_t len, int64_t k)
{
    int64_t lo = 0, hi = len - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t x = v[lo], y = v[mid], z = v[hi];
        int64_t pivot = (x < y) ? ((y < z) ? y : ((x < z) ? z : x)) : ((x < z) ? x : ((y < z) ? z : y));
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (v[i] < pivot) ++i;
            while (v[j] > pivot) --j;
            if (i <= j) {
                int64_t t = v[i];
                v[i] = v[j];
                v[j] = t;
                ++i;
                --j;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return v[k];
    }
    return v[k];
}

/*
 * Directed R-MAT graph with exactly m distinct edges and no self-loops, as a
 * CSR with rows sorted by destination.
 *
 * Draw t (t = 0, 1, 2, ...) descends `scale` = ceil(log2 n) levels, using draw
 * counter t*scale + level of the edge stream.  A draw whose source or
 * destination is >= n, or whose endpoints are equal, is rejected.  Both
 * endpoints are then relabelled by a seeded Fisher-Yates permutation, so degree
 * is not correlated with vertex id.  The graph is the set of the first m
 * distinct accepted edges in draw order.
 *
 * Returns 0 on success, 1 on invalid arguments, 2 on allocation failure.
 */
int dblgen_rmat_csr(int32_t n, int64_t m, double a, double b, double c, uint64_t seed,
                    int32_t *row_ptr, int32_t *col)
{
    if (n <= 0 || m < 0 || !row_ptr || (m > 0 && !col)) return 1;
    if ((double)m > (double)n * (double)(n - 1)) return 1;
    if (m > 0x7fffffffLL) return 1;
    int scale = 0;
    while ((1LL << scale) < (int64_t)n) ++scale;
    const double ab = a + b, abc = a + b + c;

    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!perm || !cnt) { free(perm); free(cnt); return 2; }
    make_perm(n, seed, perm);
    const uint64_t key = stream_key(seed, TAG_EDGES);

    int64_t cap = 0, nvalid = 0, ndrawn = 0;
    int32_t *src = NULL;
    uint64_t *keyv = NULL, *bucket = NULL;
    int64_t *first = NULL;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!off) { free(perm); free(cnt); return 2; }
    int64_t want = m + m / 4 + 1024;
    int rc = 0;

    for (;;) {
        /* draw `want` more edges */
        if (nvalid + want > cap) {
            int64_t ncap = nvalid + want;
            int32_t *s2 = (int32_t *)realloc(src, sizeof(int32_t) * (size_t)ncap);
            if (!s2) { rc = 2; goto done; }
            src = s2;
            uint64_t *k2 = (uint64_t *)realloc(keyv, sizeof(uint64_t) * (size_t)ncap);
            if (!k2) { rc = 2; goto done; }
            keyv = k2;
            cap = ncap;
        }
        int nth = 1;
#ifdef _OPENMP
        nth = omp_get_max_threads();
#endif
        int64_t *tcount = (int64_t *)calloc((size_t)nth + 1, sizeof(int64_t));
        if (!tcount) { rc = 2; goto done; }
        const int64_t base = ndrawn;
        /* pass 1: count accepted per thread-chunk; pass 2: write in chunk order */
        for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel num_threads(nth)
            {
                int tid = 0;
#ifdef _OPENMP
                tid = omp_get_thread_num();
#endif
                int64_t lo = base + want * tid / nth, hi = base + want * (tid + 1) / nth;
                int64_t pos = pass ? nvalid + tcount[tid] : 0;
                for (int64_t t = lo; t < hi; ++t) {
                    uint64_t s = 0, d = 0;
                    for (int lv = 0; lv < scale; ++lv) {
                        double u = unit53(sm64_at(key, (uint64_t)t * (uint64_t)scale + (uint64_t)lv));
                        uint64_t sb, db;
                        if (u < a) { sb = 0; db = 0; }
                        else if (u < ab) { sb = 0; db = 1; }
                        else if (u < abc) { sb = 1; db = 0; }
                        else { sb = 1; db = 1; }
                        s = (s << 1) | sb;
                        d = (d << 1) | db;
                    }
                    if (s >= (uint64_t)n || d >= (uint64_t)n || s == d) continue;
                    if (pass) {
                        src[pos] = perm[s];
                        keyv[pos] = ((uint64_t)perm[d] << 36) | (uint64_t)t;
                        ++pos;
                    } else {
                        ++pos;
                    }
                }
                if (!pass) tcount[tid + 1] = pos;
            }
            if (!pass)
                for (int i = 0; i < nth; ++i) tcount[i + 1] += tcount[i];
        }
        nvalid += tcount[nth];
        ndrawn += want;
        free(tcount);

        /* bucket all accepted draws by source, sort each bucket by (dst, draw) */
        memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
        for (int64_t i = 0; i < nvalid; ++i) cnt[src[i] + 1]++;
        off[0] = 0;
        for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v + 1];
        free(bucket);
        bucket = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nvalid > 0 ? nvalid : 1));
        if (!bucket) { rc = 2; goto done; }
        memcpy(cnt, off, sizeof(int64_t) * (size_t)n);
        for (int64_t i = 0; i < nvalid; ++i) bucket[cnt[src[i]]++] = keyv[i];
#pragma omp parallel for schedule(dynamic, 1024)
        for (int32_t v = 0; v < n; ++v) {
            int64_t len = off[v + 1] - off[v];
            if (len > 1) qsort(bucket + off[v], (size_t)len, sizeof(uint64_t), cmp_u64);
        }
        /* first occurrence of every distinct (src, dst) */
        int64_t uniq = 0;
#pragma omp parallel for reduction(+ : uniq) schedule(dynamic, 1024)
        for (int32_t v = 0; v < n; ++v) {
            for (int64_t i = off[v]; i < off[v + 1]; ++i)
                if (i == off[v] || (bucket[i] >> 36) != (bucket[i - 1] >> 36)) ++uniq;
        }
        if (uniq < m) {
            want = (m - uniq) * 2 + 1024;
            continue;
        }
        free(first);
        first = (int64_t *)malloc(sizeof(int64_t) * (size_t)(uniq > 0 ? uniq : 1));
        if (!first) { rc = 2; goto done; }
        int64_t f = 0;
        for (int32_t v = 0; v < n; ++v)
            for (int64_t i = off[v]; i < off[v + 1]; ++i)
                if (i == off[v] || (bucket[i] >> 36) != (bucket[i - 1] >> 36))
                    first[f++] = (int64_t)(bucket[i] & ((1ULL << 36) - 1));
        int64_t thresh = (m > 0) ? select_kth(first, uniq, m - 1) : -1;
        /* keep first occurrences drawn at or before the threshold draw */
        row_ptr[0] = 0;
        int64_t e = 0;
        for (int32_t v = 0; v < n; ++v) {
            for (int64_t i = off[v]; i < off[v + 1]; ++i) {
                if (i != off[v] && (bucket[i] >> 36) == (bucket[i - 1] >> 36)) continue;
                if ((int64_t)(bucket[i] & ((1ULL << 36) - 1)) > thresh) continue;
                col[e++] = (int32_t)(bucket[i] >> 36);
            }
            row_ptr[v + 1] = (int32_t)e;
        }
        if (e != m) rc = 3;
        break;
    }
done:
    free(perm);
    free(cnt);
    free(off);
    free(src);
    free(keyv);
    free(bucket);
    free(first);
    return rc;
}

/* ---- open-addressing set of (u, v) pairs, for the insertion stream ---- */
typedef struct {
    uint64_t *slot;
    uint64_t mask;
} pairset;

static int ps_init(pairset *s, int64_t expected)
{
    uint64_t cap = 1024;
    while (cap < (uint64_t)expected * 2) cap <<= 1;
    s->slot = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!s->slot) return 0;
    memset(s->slot, 0xff, sizeof(uint64_t) * cap);
    s->mask = cap - 1;
    return 1;
}

/* returns 1 if inserted, 0 if present */
static int ps_add(pairset *s, uint64_t k)
{
    uint64_t h = mix64(k) & s->mask;
    while (s->slot[h] != ~0ULL) {
        if (s->slot[h] == k) return 0;
        h = (h + 1) & s->mask;
    }
    s->slot[h] = k;
    return 1;
}

static int csr_has(const int32_t *row_ptr, const int32_t *col, int32_t u, int32_t v)
{
    int64_t lo = row_ptr[u], hi = (int64_t)row_ptr[u + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] == v) return 1;
        if (col[mid] < v) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0;
}

/*
 * `count` new edges (u, v), u != v, uniform over the pairs that are neither in
 * the CSR graph (rows sorted) nor earlier in the stream.  Returns 0, or 1 on
 * invalid arguments, 2 on allocation failure.
 */
int dblgen_insertions(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t count,
                      uint64_t seed, int32_t *src, int32_t *dst)
{
    if (n < 2 || count < 0 || !row_ptr) return 1;
    pairset s;
    if (!ps_init(&s, count + 16)) return 2;
    const uint64_t key = stream_key(seed, TAG_INSERT);
    uint64_t t = 0;
    for (int64_t i = 0; i < count;) {
        int32_t u = (int32_t)bounded(sm64_at(key, t++), (uint64_t)n);
        int32_t v = (int32_t)bounded(sm64_at(key, t++), (uint64_t)n);
        if (u == v || csr_has(row_ptr, col, u, v)) continue;
        if (!ps_add(&s, (uint64_t)u * (uint64_t)n + (uint64_t)v)) continue;
        src[i] = u;
        dst[i] = v;
        ++i;
    }
    free(s.slot);
    return 0;
}

/* CSR of base graph plus extra edges (rows unsorted beyond the base part). */
static int merged_csr(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t n_extra,
                      const int32_t *xs, const int32_t *xd, int64_t **rp_out, int32_t **col_out)
{
    int64_t m0 = row_ptr[n];
    int64_t *rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *cc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m0 + n_extra + 1));
    if (!rp || !cc) { free(rp); free(cc); return 0; }
    for (int32_t v = 0; v < n; ++v) rp[v + 1] = row_ptr[v + 1] - row_ptr[v];
    for (int64_t i = 0; i < n_extra; ++i) rp[xs[i] + 1]++;
    for (int32_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cur) { free(rp); free(cc); return 0; }
    for (int32_t v = 0; v < n; ++v) {
        cur[v] = rp[v];
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) cc[cur[v]++] = col[e];
    }
    for (int64_t i = 0; i < n_extra; ++i) cc[cur[xs[i]]++] = xd[i];
    free(cur);
    *rp_out = rp;
    *col_out = cc;
    return 1;
}

/*
 * Mixed query stream of q pairs on the graph G + extra edges.
 * Even index i: (u, v) uniform and independent.
 * Odd index i: u uniform with at least one out-edge, v a descendant of u other
 * than u.  exact=1: v uniform over Des(u)\{u} by a full BFS.  exact=0: v is the
 * end of a random forward walk of U[1,32] steps that stops early at a vertex
 * with no out-edges (retried up to 8 times while it ends at u).
 * Every query draws from its own counter range, so the stream is identical for
 * any thread count.  Returns 0, 1 on invalid arguments, 2 on allocation failure.
 */
int dblgen_queries(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t n_extra,
                   const int32_t *xs, const int32_t *xd, int64_t q, uint64_t seed, int exact,
                   int32_t *qu, int32_t *qv)
{
    if (n < 1 || q < 0 || !row_ptr) return 1;
    int64_t *rp;
    int32_t *cc;
    if (!merged_csr(n, row_ptr, col, n_extra, xs, xd, &rp, &cc)) return 2;
    const uint64_t key = stream_key(seed, TAG_QUERY);
    int rc = 0;
#pragma omp parallel
    {
        int32_t *stamp = NULL, *queue = NULL;
        if (exact) {
            stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
            queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
            if (!stamp || !queue) {
#pragma omp atomic write
                rc = 2;
            } else {
                for (int32_t i = 0; i < n; ++i) stamp[i] = -1;
            }
        }
        int32_t epoch = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < q; ++i) {
            uint64_t base = (uint64_t)i << 20, t = 0;
            if (rc) continue;
            if ((i & 1) == 0) {
                qu[i] = (int32_t)bounded(sm64_at(key, base + t++), (uint64_t)n);
                qv[i] = (int32_t)bounded(sm64_at(key, base + t++), (uint64_t)n);
                continue;
            }
            int32_t u = -1, v = -1;
            for (int attempt = 0; attempt < (1 << 16) && v < 0; ++attempt) {
                u = (int32_t)bounded(sm64_at(key, base + t++), (uint64_t)n);
                if (rp[u + 1] == rp[u]) continue;
                if (exact) {
                    ++epoch;
                    int64_t head = 0, tail = 0;
                    stamp[u] = epoch;
                    queue[tail++] = u;
                    while (head < tail) {
                        int32_t w = queue[head++];
                        for (int64_t e = rp[w]; e < rp[w + 1]; ++e) {
                            int32_t x = cc[e];
                            if (stamp[x] != epoch) {
                                stamp[x] = epoch;
                                queue[tail++] = x;
                            }
                        }
                    }
                    /* queue[1..tail) is Des(u)\{u} */
                    if (tail > 1)
                        v = queue[1 + (int64_t)bounded(sm64_at(key, base + t++), (uint64_t)(tail - 1))];
                } else {
                    for (int tries = 0; tries < 8 && v < 0; ++tries) {
                        int steps = 1 + (int)bounded(sm64_at(key, base + t++), 32);
                        int32_t x = u;
                        for (int s = 0; s < steps; ++s) {
                            int64_t deg = rp[x + 1] - rp[x];
                            if (deg == 0) break;
                            x = cc[rp[x] + (int64_t)bounded(sm64_at(key, base + t++), (uint64_t)deg)];
                        }
                        if (x != u) v = x;
                    }
                }
            }
            if (v < 0) { /* graph without any out-edges: fall back to a uniform pair */
                v = (int32_t)bounded(sm64_at(key, base + t++), (uint64_t)n);
            }
            qu[i] = u;
            qv[i] = v;
        }
        free(stamp);
        free(queue);
    }
    free(rp);
    free(cc);
    return rc;
}

/*
 * Batch sizes floor(exp(U[ln lo, ln(hi+1)))), clamped to [lo, hi], drawn until
 * they sum to `total` (the last one is cut).  Returns the number of batches
 * written to sizes[0..cap), or -1 if cap is too small.
 */
int64_t dblgen_loguniform_batches(int64_t total, int64_t lo, int64_t hi, uint64_t seed,
                                  int64_t *sizes, int64_t cap)
{
    const uint64_t key = stream_key(seed, TAG_SIZES);
    double l0 = log((double)lo), l1 = log((double)hi + 1.0);
    int64_t done = 0, nb = 0;
    uint64_t t = 0;
    while (done < total) {
        if (nb >= cap) return -1;
        double u = unit53(sm64_at(key, t++));
        int64_t s = (int64_t)exp(l0 + (l1 - l0) * u);
        if (s < lo) s = lo;
        if (s > hi) s = hi;
        if (s > total - done) s = total - done;
        sizes[nb++] = s;
        done += s;
    }
    return nb;
}
