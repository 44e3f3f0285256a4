// Batched edge insertion and label repair (Section 5).
//
// Appending: each vertex keeps its inserted out-edges (and in-edges) in one
// contiguous segment of an edge pool, (offset, length, capacity), grown by
// doubling; a batch counts edges per vertex, grows the segments that
// overflow (old segments are abandoned, so snapshots stay valid), and writes
// the new ids.  The pool never holds more than 4 entries per stored edge.
//
// Repair: Algorithm 3 skips an edge (u, v) when DL_out(u) and DL_in(v) already
// intersect (u already reaches v, so no label changes).  Otherwise its BFS from
// v adds DL_in(u) to every descendant, and the mirror adds DL_out(v) to every
// ancestor of u; BL_in / BL_out the same.  Here the seed step ORs fwd(u) into
// fwd(v) and bwd(v) into bwd(u) for every edge of the batch, and the ordinary
// propagation (which sees the appended edges) carries the change to the
// fixpoint: the result equals one-by-one insertion in any order.
#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_kernels.cuh"
#include "dbl_persistent.cuh"

namespace dbl {

__global__ void k_ins_validate(const int32_t *src, const int32_t *dst, int64_t b, int32_t n, uint32_t *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        if ((uint32_t)src[i] >= (uint32_t)n || (uint32_t)dst[i] >= (uint32_t)n) set_status(status, DBL_ERR_INVALID);
    }
}

// per-edge rank inside its source (out) and destination (in) vertex batch
// Every mutating kernel of an insertion first reads the status word: after a
// failed validation (or any latched error) it changes nothing, so the
// asynchronous form needs no host round trip between validation and append.
__device__ __forceinline__ bool status_set(const uint32_t *status) { return *(const volatile uint32_t *)status != 0; }

__global__ void k_ins_count(const int32_t *src, const int32_t *dst, int64_t b, int32_t *cnt_out, int32_t *cnt_in,
                            int32_t *pos_out, int32_t *pos_in, unsigned long long *stats, const uint32_t *status,
                            uint32_t *dirty)
{
    if (status_set(status)) return;
    unsigned long long loops = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[i], v = dst[i];
        if (u == v) {
            pos_out[i] = -1;
            pos_in[i] = -1;
            ++loops;
            continue;
        }
        pos_out[i] = atomicAdd(cnt_out + u, 1);
        pos_in[i] = atomicAdd(cnt_in + v, 1);
        mark_dirty(dirty, u);  // both endpoints' adjacency metadata change
        mark_dirty(dirty, v);
    }
    if (loops) atomicAdd(stats + 13, loops);
}

__device__ __forceinline__ int32_t grown_cap(int32_t need)
{
    int32_t c = 4;
    while (c < need) c <<= 1;
    return c;
}

// The first edge of each vertex batch grows that vertex's segment if needed.
// New segments are reserved with one atomicAdd per warp (a warp-wide prefix
// sum of the sizes) instead of one per vertex on the shared pool top.
__global__ void k_ins_grow(const int32_t *src, const int32_t *dst, int64_t b, const int32_t *cnt_out,
                           const int32_t *cnt_in, const int32_t *pos_out, const int32_t *pos_in, VMeta *vm,
                           int32_t *pool_out, int32_t *pool_in, int64_t *pool_top, int64_t pool_cap,
                           uint32_t *status)
{
    if (status_set(status)) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < b; base += stride) {
        const int64_t i = base + threadIdx.x;
        for (int dir = 0; dir < 2; ++dir) {
            int32_t x = 0, len = 0, nc = 0;
            VAdj a{0, 0u, 0, 0};
            if (i < b && (dir ? pos_in[i] : pos_out[i]) == 0) {
                x = dir ? dst[i] : src[i];
                a = load_vadj(vm, dir, x);
                len = a.len;
                const int32_t need = len + (dir ? cnt_in[x] : cnt_out[x]);
                if (need > va_cap(a.dc)) nc = grown_cap(need);
            }
            unsigned long long incl = (unsigned long long)nc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned long long total = __shfl_sync(kFull, incl, 31);
            if (total == 0) continue;
            unsigned long long wbase = 0;
            if (lane == 31) wbase = atomicAdd((unsigned long long *)(pool_top + dir), total);
            wbase = __shfl_sync(kFull, wbase, 31);
            if (!nc) continue;
            const long long off = (long long)(wbase + incl - (unsigned long long)nc);
            if (off + nc > pool_cap) {
                set_status(status, DBL_ERR_CAPACITY);  // cannot happen: pool holds 4x the edge capacity
                continue;
            }
            int32_t *pool = dir ? pool_in : pool_out;
            for (int32_t j = 0; j < len; ++j) pool[off + j] = pool[a.off + j];
            vm[x].d[dir].off = (int32_t)off;
            vm[x].d[dir].dc = va_dc(va_deg(a.dc), nc);
        }
    }
}

__global__ void k_ins_write(const int32_t *src, const int32_t *dst, int64_t b, const int32_t *pos_out,
                            const int32_t *pos_in, const VMeta *vm, int32_t *pool_out, int32_t *pool_in,
                            const uint32_t *status)
{
    if (status_set(status)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t po = pos_out[i];
        if (po < 0) continue;
        const int32_t u = src[i], v = dst[i], pi = pos_in[i];
        const VAdj au = load_vadj(vm, 0, u), av = load_vadj(vm, 1, v);
        // a segment that could not grow (pool exhausted, status already set) is not written past its end
        if (au.len + po < va_cap(au.dc)) pool_out[(int64_t)au.off + au.len + po] = v;
        if (av.len + pi < va_cap(av.dc)) pool_in[(int64_t)av.off + av.len + pi] = u;
    }
}

__global__ void k_ins_commit(const int32_t *src, const int32_t *dst, int64_t b, int32_t *cnt_out, int32_t *cnt_in,
                             const int32_t *pos_out, const int32_t *pos_in, VMeta *vm, const uint32_t *status)
{
    if (status_set(status)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        if (pos_out[i] == 0) {
            const int32_t u = src[i];
            vm[u].d[0].len += cnt_out[u];
            cnt_out[u] = 0;
        }
        if (pos_in[i] == 0) {
            const int32_t v = dst[i];
            vm[v].d[1].len += cnt_in[v];
            cnt_in[v] = 0;
        }
    }
}

// Seeds of the repair: the skip test of Algorithm 3, then fwd(v) |= fwd(u),
// bwd(u) |= bwd(v); changed endpoints start the frontier.
template <int HS, int WD>
__device__ __forceinline__ void seed_edges(const int32_t *src, const int32_t *dst, int64_t b, const DevGraph &g,
                                           uint64_t *rec, uint64_t dlm, const FrontierOut &f,
                                           unsigned long long *stats);

template <int HS, int WD>
__global__ void __launch_bounds__(kBlock) k_ins_seed(const int32_t *src, const int32_t *dst, int64_t b, DevGraph g,
                                                     uint64_t *rec, uint64_t dlm, FrontierOut f,
                                                     unsigned long long *stats)
{
    if (status_set(f.status)) return;
    seed_edges<HS, WD>(src, dst, b, g, rec, dlm, f, stats);
}

// One edge's seed: Algorithm 3's skip test on DL_out(u) and DL_in(v), then
// fwd(v) |= fwd(u) and bwd(u) |= bwd(v).  All four half-records are loaded at
// once (one memory round trip).  Returns true if the edge was applied;
// want_f / want_b say whether fwd(v) / bwd(u) gained bits.  That is decided
// from the values loaded before the ORs, which are then fire-and-forget: the
// first OR that adds a bit to a word was issued by a thread whose load did not
// see that bit, and a load that misses bits the OR brings means the word
// grows.  Callers read the frontier only after a grid barrier or a launch.
template <int HS, int WD>
__device__ __forceinline__ bool seed_one(int32_t u, int32_t v, uint64_t *rec, uint32_t *dirty, uint64_t dlm,
                                         bool &want_f, bool &want_b)
{
    constexpr int RW = 2 * HS;
    uint64_t *fu = rec + (size_t)u * RW, *bu = fu + HS;
    uint64_t *fv = rec + (size_t)v * RW, *bv = fv + HS;
    uint64_t a[HS], c[HS], x[HS], y[HS];
    if constexpr (HS == 2) {  // 32-byte records: one load per record
        load_rec32(fu, x[0], x[1], a[0], a[1]);
        load_rec32(fv, c[0], c[1], y[0], y[1]);
    } else if constexpr (HS == 1) {  // packed 16-byte records: one load per record
        const ulonglong2 ru = __ldcg(reinterpret_cast<const ulonglong2 *>(fu));
        const ulonglong2 rv = __ldcg(reinterpret_cast<const ulonglong2 *>(fv));
        x[0] = ru.x;
        a[0] = ru.y;
        c[0] = rv.x;
        y[0] = rv.y;
    } else {
        load_half<HS>(bu, a);  // DL_out(u) | BL_out(u)
        load_half<HS>(fv, c);  // DL_in(v)  | BL_in(v)
        load_half<HS>(fu, x);  // DL_in(u)  | BL_in(u)
        load_half<HS>(bv, y);  // DL_out(v) | BL_out(v)
    }
    uint64_t inter = 0;
    if constexpr (WD == 0) {
        inter = a[0] & c[0] & dlm;  // packed: the DL bits of the one word
    } else {
#pragma unroll
        for (int w = 0; w < WD; ++w) inter |= a[w] & c[w];
    }
    if (inter) return false;
#pragma unroll
    for (int w = 0; w < HS; ++w) {
        if (x[w] & ~c[w]) {
            atomicOr((unsigned long long *)(fv + w), x[w]);
            want_f = true;
        }
        if (y[w] & ~a[w]) {
            atomicOr((unsigned long long *)(bu + w), y[w]);
            want_b = true;
        }
    }
    if (want_f) mark_dirty(dirty, v);
    if (want_b) mark_dirty(dirty, u);
    return true;
}

template <int HS, int WD>
__device__ __forceinline__ void seed_edges(const int32_t *src, const int32_t *dst, int64_t b, const DevGraph &g,
                                           uint64_t *rec, uint64_t dlm, const FrontierOut &f,
                                           unsigned long long *stats)
{
    unsigned long long skipped = 0, applied = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < b; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool want_f = false, want_b = false;
        int32_t u = 0, v = 0;
        if (i < b) {
            u = src[i];
            v = dst[i];
            if (u != v) {
                if (seed_one<HS, WD>(u, v, rec, g.dirty, dlm, want_f, want_b)) ++applied;
                else ++skipped;
            }
        }
        warp_enqueue(want_f, v, 0, g, f);
        warp_enqueue(want_b, u, 1, g, f);
    }
    warp_stat_add(stats, 12, skipped);
    warp_stat_add(stats, 11, applied);
}

// ---------------------------------------------------------------------------
// Whole insertion batch in one cooperative launch (persistent form), with a
// grid barrier after each phase:
//   P1 validate + count: each edge takes its slot straight from the live
//      segment length (atomicAdd on len, so no commit pass is needed); if an
//      id is invalid the slots are given back and the launch ends
//   P2 seed + grow: each edge applies its seed (skip test, endpoint ORs);
//      whether fwd(v) / bwd(u) gained bits is kept in bit 30 of the edge's
//      slot words (slots are < 2^29); the one edge whose slot equals the old
//      capacity grows the segment (copying the old capacity's worth of
//      entries; the batch's own entries are written after the barrier)
//   P3 write + enqueue: the batch's ids go into their slots, and the changed
//      endpoints form the level-0 frontier (tasks resolved against the final
//      segment offsets and lengths)
//   P4 propagation levels, as in k_propagate_persistent.
// Seeding before the appended edges are visible is sound: seeds read and OR
// labels only, and the first level that walks adjacency runs after P3.  A
// failed validation leaves the index as it was.
constexpr int32_t kWantBit = 1 << 30;

// The batches one launch applies together: batch j's edges are
// src[j][0..len), dst[j][0..len), at positions off[j] .. off[j + 1) of the
// launch's edge range.  Batches queued with no call that reads the index
// between them are applied as one (the labels are the unique fixpoint of the
// graph with all of them, whatever the grouping).
constexpr int kMaxGroup = 32;
struct BatchList {
    int32_t nb;
    int64_t off[kMaxGroup + 1];
    const int32_t *src[kMaxGroup];
    const int32_t *dst[kMaxGroup];
};

struct InsArgs {
    const int32_t *src, *dst;  // the edges when nb == 1
    BatchList bl;
    int64_t b;
    int32_t n;
    VMeta *vm;
    int32_t *pool_out, *pool_in;
    int64_t *pool_top;
    int64_t pool_cap;
    int32_t *slot_out, *slot_in;
    DevGraph g;
    uint64_t *rec;
    FTask *f0, *f1;
    uint32_t *c3;
    int64_t cap;
    uint32_t *mark;  // frontier bitmaps, parity 0 then 1 (2 * wpd words each)
    int64_t wpd;
    unsigned long long *stats;
    uint32_t *status;
    uint32_t *bad;   // this batch has an invalid id (zero before the launch)
    uint32_t *grow;  // some segment of this batch must grow (zero before the launch)
    uint64_t dlm;    // packed labels: the DL bits of a half word
};

// Edge i of the launch's batches.
__device__ __forceinline__ void edge_at(const InsArgs &a, int64_t i, int32_t &u, int32_t &v)
{
    if (a.bl.nb <= 1) {
        u = a.src[i];
        v = a.dst[i];
        return;
    }
    int lo = 0, hi = a.bl.nb - 1;  // the batch j with off[j] <= i < off[j + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.bl.off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int64_t k = i - a.bl.off[lo];
    u = a.bl.src[lo][k];
    v = a.bl.dst[lo][k];
}

// Adjacency metadata of one direction from a VMeta sector loaded as four words.
__device__ __forceinline__ VAdj vadj_of_words(uint64_t lo, uint64_t hi)
{
    return VAdj{(int32_t)(uint32_t)lo, (uint32_t)(lo >> 32), (int32_t)(uint32_t)hi, (int32_t)(uint32_t)(hi >> 32)};
}

// edges per lane in flight at each stage of the repair's flattened levels
constexpr int kInsUnroll = 1;

template <int HS, int WD, int TEAM>
__device__ __forceinline__ void insert_phases(const InsArgs &a, GridSync &gs, const Stage &st, int64_t max_levels)
{
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    const int lane = threadIdx.x & 31;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    // a status latched before this launch (asynchronous form) leaves every
    // phase empty; no block writes the status word before the first barrier,
    // so all blocks read the same value here
    if (ld_volatile_u32(a.status)) return;
    // P1: validate and count: each edge takes its slots from the live segment
    // lengths (atomicAdd on len, so no commit pass is needed); an invalid id
    // raises the batch's own flag, and then every slot taken is given back
    // after the barrier and nothing else changes.  The segments' capacities
    // are read in the same round trip (no segment grows in this phase): a slot
    // at or past its segment's capacity raises the batch's grow flag.
    bool grow_any;
    {
        unsigned long long loops = 0;
        bool grow = false;
        for (int64_t i = t0; i < a.b; i += nt) {
            int32_t u, v;
            edge_at(a, i, u, v);
            if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
                atomicExch(a.bad, 1u);
                a.slot_out[i] = a.slot_in[i] = -1;
                continue;
            }
            if (u == v) {
                a.slot_out[i] = a.slot_in[i] = -1;
                ++loops;
                continue;
            }
            const int32_t so = atomicAdd(&a.vm[u].d[0].len, 1);
            const int32_t si = atomicAdd(&a.vm[v].d[1].len, 1);
            const uint32_t dcu = __ldcg(&a.vm[u].d[0].dc), dcv = __ldcg(&a.vm[v].d[1].dc);
            a.slot_out[i] = so;
            a.slot_in[i] = si;
            grow |= so >= va_cap(dcu) || si >= va_cap(dcv);
            mark_dirty(a.g.dirty, u);
            mark_dirty(a.g.dirty, v);
        }
        if (__any_sync(kFull, grow) && lane == 0) atomicOr(a.grow, 1u);
        if (leader) a.c3[0] = a.c3[1] = a.c3[2] = 0;
        if (!gs.sync(a.status)) return;
        if (ld_volatile_u32(a.bad)) {
            for (int64_t i = t0; i < a.b; i += nt) {
                if (a.slot_out[i] < 0) continue;
                int32_t u, v;
                edge_at(a, i, u, v);
                atomicSub(&a.vm[u].d[0].len, 1);
                atomicSub(&a.vm[v].d[1].len, 1);
            }
            if (!gs.sync(a.status)) return;  // every block has read the flags
            if (leader) {
                *(volatile uint32_t *)a.bad = 0;
                *(volatile uint32_t *)a.grow = 0;
                set_status(a.status, DBL_ERR_INVALID);
            }
            return;
        }
        grow_any = ld_volatile_u32(a.grow) != 0;  // the same for every block
        warp_stat_add(a.stats, 13, loops);
    }
    if (!grow_any) {
        // P2 (no segment grows): seeds, the batch's ids into their slots, and
        // the level-0 frontier, in one phase.  Lengths are final and no
        // segment moves, so each endpoint's metadata sector (both directions,
        // one load) gives both where its id goes and the task's edge range.
        FrontierOut f{a.f0, a.c3, a.cap, a.mark, a.wpd, a.status};  // level-0 frontier: parity 0
        unsigned long long skipped = 0, applied = 0;
        for (int64_t wbase = (int64_t)blockIdx.x * blockDim.x; wbase < a.b; wbase += nt) {  // block-uniform
            const int64_t i = wbase + threadIdx.x;
            bool want_f = false, want_b = false;
            int32_t u = 0, v = 0;
            VAdj eu{0, 0u, 0, 0}, ev{0, 0u, 0, 0};
            if (i < a.b) {
                const int32_t so = a.slot_out[i], si = a.slot_in[i];
                edge_at(a, i, u, v);
                if (so >= 0) {
                    uint64_t mu[4], mv[4];
                    load_rec32(reinterpret_cast<const uint64_t *>(a.vm + u), mu[0], mu[1], mu[2], mu[3]);
                    load_rec32(reinterpret_cast<const uint64_t *>(a.vm + v), mv[0], mv[1], mv[2], mv[3]);
                    if (seed_one<HS, WD>(u, v, a.rec, a.g.dirty, a.dlm, want_f, want_b)) ++applied;
                    else ++skipped;
                    const VAdj au = vadj_of_words(mu[0], mu[1]), av = vadj_of_words(mv[2], mv[3]);
                    eu = vadj_of_words(mu[2], mu[3]);  // u's in-edges: bwd(u) changed
                    ev = vadj_of_words(mv[0], mv[1]);  // v's out-edges: fwd(v) changed
                    a.pool_out[(int64_t)au.off + so] = v;
                    a.pool_in[(int64_t)av.off + si] = u;
                }
            }
            stage_enqueue_at(want_f, v, 0, AdjRange{ev.start, va_deg(ev.dc), ev.off, ev.len}, f, st);
            stage_enqueue_at(want_b, u, 1, AdjRange{eu.start, va_deg(eu.dc), eu.off, eu.len}, f, st);
        }
        stage_flush(f, st);
        warp_stat_add(a.stats, 12, skipped);
        warp_stat_add(a.stats, 11, applied);
        if (!gs.sync(a.status)) return;
        if (leader) *(volatile uint32_t *)a.grow = 0;  // every block read it before this barrier
    } else {
    // P2: seeds (Algorithm 3's skip test, then the endpoint ORs; whether
    // fwd(v) / bwd(u) gained bits is kept in bit 30 of the edge's slot words,
    // slots being < 2^29), and growth of the segments that overflowed: both
    // directions' metadata are read in one round trip and the pool is reserved
    // once per block for both
    {
        __shared__ unsigned long long s_woff[2][32];  // per-warp growth, then its offset in the block's range
        __shared__ unsigned long long s_gbase[2];
        const int warp = threadIdx.x >> 5, nwb = blockDim.x >> 5;
        unsigned long long skipped = 0, applied = 0;
        for (int64_t wbase = (int64_t)blockIdx.x * blockDim.x; wbase < a.b; wbase += nt) {  // block-uniform
            const int64_t i = wbase + threadIdx.x;
            int32_t x[2] = {0, 0}, old_cap[2] = {0, 0}, nc[2] = {0, 0};
            VAdj ad[2] = {{0, 0u, 0, 0}, {0, 0u, 0, 0}};
            if (i < a.b) {
                const int32_t sw[2] = {a.slot_out[i], a.slot_in[i]};
                edge_at(a, i, x[0], x[1]);
                // with 16-byte halves the segment metadata is loaded before the
                // seed's records, in the same round trip (len is final after the
                // count phase); wider records leave no registers for that
                constexpr bool kEarly = HS <= 2;
                if (kEarly) {
#pragma unroll
                    for (int dir = 0; dir < 2; ++dir)
                        if (sw[dir] >= 0) ad[dir] = load_vadj(a.vm, dir, x[dir]);
                }
                if (sw[0] >= 0) {
                    bool want_f = false, want_b = false;
                    if (seed_one<HS, WD>(x[0], x[1], a.rec, a.g.dirty, a.dlm, want_f, want_b)) ++applied;
                    else ++skipped;
                    if (want_b) a.slot_out[i] = sw[0] | kWantBit;
                    if (want_f) a.slot_in[i] = sw[1] | kWantBit;
                }
#pragma unroll
                for (int dir = 0; dir < 2; ++dir) {
                    if (sw[dir] < 0) continue;
                    if (!kEarly) ad[dir] = load_vadj(a.vm, dir, x[dir]);
                    old_cap[dir] = va_cap(ad[dir].dc);
                    if (sw[dir] == old_cap[dir]) nc[dir] = grown_cap(ad[dir].len);
                }
            }
            unsigned long long incl[2];
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                incl[dir] = (unsigned long long)nc[dir];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long t = __shfl_up_sync(kFull, incl[dir], o);
                    if (lane >= o) incl[dir] += t;
                }
                if (lane == 31) s_woff[dir][warp] = incl[dir];
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                const int dir = threadIdx.x;
                unsigned long long run = 0;
                for (int w = 0; w < nwb; ++w) {
                    const unsigned long long t = s_woff[dir][w];
                    s_woff[dir][w] = run;
                    run += t;
                }
                s_gbase[dir] = run ? atomicAdd((unsigned long long *)(a.pool_top + dir), run) : 0ull;
            }
            __syncthreads();
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                if (!nc[dir]) continue;
                const long long off =
                    (long long)(s_gbase[dir] + s_woff[dir][warp] + incl[dir] - (unsigned long long)nc[dir]);
                if (off + nc[dir] > a.pool_cap) {
                    set_status(a.status, DBL_ERR_CAPACITY);  // cannot happen: the pool holds 4x the edge capacity
                    continue;
                }
                int32_t *pool = dir ? a.pool_in : a.pool_out;
                for (int32_t j = 0; j < old_cap[dir]; ++j) pool[off + j] = pool[ad[dir].off + j];
                a.vm[x[dir]].d[dir].off = (int32_t)off;
                a.vm[x[dir]].d[dir].dc = va_dc(va_deg(ad[dir].dc), nc[dir]);
            }
            __syncthreads();  // s_woff is reused by the next round
        }
        warp_stat_add(a.stats, 12, skipped);
        warp_stat_add(a.stats, 11, applied);
    }
    if (!gs.sync(a.status)) return;
    if (leader) *(volatile uint32_t *)a.grow = 0;  // every block read it before this barrier
    // P3: write the batch's ids into their slots, and enqueue the seeds'
    // changed endpoints (their tasks carry the final adjacency locations)
    {
        FrontierOut f{a.f0, a.c3, a.cap, a.mark, a.wpd, a.status};  // level-0 frontier: parity 0
        for (int64_t wbase = (int64_t)blockIdx.x * blockDim.x; wbase < a.b; wbase += nt) {  // block-uniform
            const int64_t i = wbase + threadIdx.x;
            bool want_f = false, want_b = false;
            int32_t u = 0, v = 0;
            VAdj eu{0, 0u, 0, 0}, ev{0, 0u, 0, 0};  // adjacency of the tasks to enqueue
            if (i < a.b) {
                const int32_t so = a.slot_out[i], si = a.slot_in[i];
                edge_at(a, i, u, v);
                if (so >= 0) {
                    want_b = (so & kWantBit) != 0;
                    want_f = (si & kWantBit) != 0;
                    const int32_t po = so & ~kWantBit, pi = si & ~kWantBit;
                    // both halves of each endpoint's metadata sector in one round trip
                    const VAdj au = load_vadj(a.vm, 0, u), av = load_vadj(a.vm, 1, v);
                    if (want_f) ev = load_vadj(a.vm, 0, v);
                    if (want_b) eu = load_vadj(a.vm, 1, u);
                    if (po < va_cap(au.dc)) a.pool_out[(int64_t)au.off + po] = v;
                    if (pi < va_cap(av.dc)) a.pool_in[(int64_t)av.off + pi] = u;
                }
            }
            // fwd(v) changed: v's out-edges (dir 0); bwd(u) changed: u's in-edges (dir 1)
            stage_enqueue_at(want_f, v, 0, AdjRange{ev.start, va_deg(ev.dc), ev.off, ev.len}, f, st);
            stage_enqueue_at(want_b, u, 1, AdjRange{eu.start, va_deg(eu.dc), eu.off, eu.len}, f, st);
        }
        stage_flush(f, st);
    }
    if (!gs.sync(a.status)) return;
    }  // P2 and P3 when a segment grows
    // P4: propagation levels
    const int64_t warp0 = t0 >> 5, nwarps = nt >> 5;
    int64_t L = 0;
    for (;; ++L) {
        const uint32_t ntk = ld_volatile_u32(a.c3 + L % 3);
        if (ntk == 0 || ld_volatile_u32(a.status)) break;
        if (L >= max_levels) {
            set_status(a.status, DBL_ERR_TIMEOUT);
            break;
        }
        if (leader) a.c3[(L + 2) % 3] = 0;
        uint32_t *cur_mark = a.mark + (size_t)(L & 1) * 2 * (size_t)a.wpd;
        uint32_t *nxt_mark = a.mark + (size_t)((L + 1) & 1) * 2 * (size_t)a.wpd;
        FrontierOut f{(L & 1) ? a.f0 : a.f1, a.c3 + (L + 1) % 3, a.cap, nxt_mark, a.wpd, a.status};
        expand_level<HS, TEAM, kInsUnroll>(a.g, RecView{a.rec, 2 * HS, HS}, (L & 1) ? a.f1 : a.f0, ntk, cur_mark, f,
                                           a.stats, warp0, nwarps, st);
        if (!gs.sync(a.status)) break;
    }
    if (leader) a.stats[8] += (unsigned long long)L;
}

template <int HS, int WD, int TEAM>
__global__ void __launch_bounds__(pblock_of(HS), 1) k_insert_persistent(InsArgs a, GridBarrier bar, int64_t max_levels)
{
    GridSync gs(bar);
    DBL_BLOCK_STAGE(st);
    insert_phases<HS, WD, TEAM>(a, gs, st, max_levels);
    gs.leave();
}

template <int HS, int WD, int TEAM>
static dbl_status launch_insert_persistent(dbl_index *ix, const InsArgs &args, cudaStream_t s)
{
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_insert_persistent<HS, WD, TEAM>, pblock_of(HS),
                                                      0);
    if (blocks_per_sm < 1) return fail(ix, DBL_ERR_CUDA, "persistent insert: kernel does not fit on an SM");
    InsArgs a = args;
    GridBarrier bar = grid_barrier_at(ix->d_counts);
    if (ix->opt.flags & DBL_FLAG_TIMING) bar.trace = ix->d_trace;
    int64_t max_levels = (int64_t)ix->n + 2;
    void *kargs[] = {&a, &bar, &max_levels};
    dim3 grid((unsigned)num_sms()), block(pblock_of(HS));
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_insert_persistent<HS, WD, TEAM>, grid, block, kargs, 0, s);
    ++ix->launches;
    return e ? cuda_fail(ix, e, "persistent insert launch") : DBL_OK;
}

template <int HS, int WD>
static dbl_status launch_insert_persistent_team(dbl_index *ix, const InsArgs &a, cudaStream_t s)
{
    switch (ix->opt.team) {
    case 1: return launch_insert_persistent<HS, WD, 1>(ix, a, s);
    case 4: return launch_insert_persistent<HS, WD, 4>(ix, a, s);
    case 16: return launch_insert_persistent<HS, WD, 16>(ix, a, s);
    case 32: return launch_insert_persistent<HS, WD, 32>(ix, a, s);
    default: return launch_insert_persistent<HS, WD, 8>(ix, a, s);
    }
}

// One cooperative launch applying the batches of `bl` (b edges in all) with
// per-edge scratch pos_out / pos_in (b entries each).  The caller accounts
// for the stored edges.
static dbl_status insert_persistent_list(dbl_index *ix, const BatchList &bl, const int32_t *src, const int32_t *dst,
                                         int64_t b, int32_t *pos_out, int32_t *pos_in, cudaStream_t s)
{
    InsArgs a;
    a.src = src;
    a.dst = dst;
    a.bl = bl;
    a.b = b;
    a.n = ix->n;
    a.vm = ix->vm;
    a.pool_out = ix->pool_out;
    a.pool_in = ix->pool_in;
    a.pool_top = ix->d_pool_top;
    a.pool_cap = ix->pool_cap;
    a.slot_out = pos_out;
    a.slot_in = pos_in;
    a.g = dev_graph(ix);
    a.rec = ix->rec;
    a.f0 = ix->front[0];
    a.f1 = ix->front[1];
    a.c3 = ix->d_counts + kCntP0;
    a.cap = ix->front_cap;
    a.mark = ix->mark;
    a.wpd = ix->wpd;
    a.stats = ix->d_stats;
    a.status = ix->d_status;
    a.bad = ix->d_counts + kCntBad;
    a.grow = ix->d_counts + kCntGrow;
    a.dlm = ix->dl_mask;
    tbegin(ix, DBL_KERNEL_PROPAGATE, s);
    dbl_status st;
    switch (ix->packed ? 0 : ix->hs * 16 + ix->wd) {
    case 0: st = launch_insert_persistent_team<1, 0>(ix, a, s); break;
    case 2 * 16 + 1: st = launch_insert_persistent_team<2, 1>(ix, a, s); break;
    case 4 * 16 + 1: st = launch_insert_persistent_team<4, 1>(ix, a, s); break;
    case 4 * 16 + 2: st = launch_insert_persistent_team<4, 2>(ix, a, s); break;
    case 8 * 16 + 1: st = launch_insert_persistent_team<8, 1>(ix, a, s); break;
    case 8 * 16 + 2: st = launch_insert_persistent_team<8, 2>(ix, a, s); break;
    case 8 * 16 + 4: st = launch_insert_persistent_team<8, 4>(ix, a, s); break;
    default: st = fail(ix, DBL_ERR_INVALID, "insert: unsupported label width");
    }
    tend(ix, s);
    return st;
}

static dbl_status insert_persistent(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, int32_t *pos_out,
                                    int32_t *pos_in, cudaStream_t s)
{
    BatchList bl;
    bl.nb = 1;
    bl.off[0] = 0;
    bl.off[1] = b;
    bl.src[0] = src;
    bl.dst[0] = dst;
    dbl_status st = insert_persistent_list(ix, bl, src, dst, b, pos_out, pos_in, s);
    if (st) return st;
    ix->edges_stored += b;
    atomic_add_host_stat(ix, 15, (uint64_t)b, s);
    if (ix->opt.flags & DBL_FLAG_ASYNC) return DBL_OK;  // errors latch; dbl_sync reports them
    dbl_status ds = read_status(ix, s);
    if (ds == DBL_ERR_INVALID) {
        ix->edges_stored -= b;  // the kernel changed nothing
        return fail(ix, ds, "insert: vertex id out of range");
    }
    return ds;
}

// Deferred insertion (DBL_FLAG_DEFER with persistent, asynchronous calls):
// dbl_insert_edges only queues the batch; the queue is applied in one
// launch by the next call that reads or changes the index otherwise (or
// when kMaxGroup batches wait).  Every query therefore observes exactly the
// insertions queued before it.
bool deferring(const dbl_index *ix)
{
    const int32_t f = ix->opt.flags;
    return (f & DBL_FLAG_DEFER) && (f & DBL_FLAG_PERSISTENT) && (f & DBL_FLAG_ASYNC);
}

static dbl_status ensure_ins_scratch(dbl_index *ix, int64_t b, cudaStream_t s)
{
    if (b <= ix->ins_bcap) return DBL_OK;
    if (ix->ins_pos) free_buf(ix, ix->ins_pos, s);
    ix->ins_pos = nullptr;
    ix->ins_bcap = 0;  // a failed allocation below leaves nothing to reuse
    int64_t nb = b < (1 << 16) ? (1 << 16) : b;
    dbl_status st = alloc_buf(ix, (void **)&ix->ins_pos, sizeof(int32_t) * 2 * (size_t)nb, s);
    if (st) return st;
    ix->ins_bcap = nb;
    return DBL_OK;
}

dbl_status flush_insertions(dbl_index *ix, cudaStream_t s)
{
    if (ix->pending.empty()) return DBL_OK;
    BatchList bl;
    bl.nb = (int32_t)ix->pending.size();
    int64_t total = 0;
    for (int j = 0; j < bl.nb; ++j) {
        bl.off[j] = total;
        bl.src[j] = ix->pending[j].src;
        bl.dst[j] = ix->pending[j].dst;
        total += ix->pending[j].b;
    }
    bl.off[bl.nb] = total;
    ix->pending.clear();
    ix->pending_edges = 0;
    // the queue's scratch was sized when its batches were queued
    const dbl_status st =
        insert_persistent_list(ix, bl, bl.src[0], bl.dst[0], total, ix->ins_pos, ix->ins_pos + ix->ins_bcap, s);
    // host-form staging buffers of the queued batches are free once this launch is done
    for (int k = 0; k < ix->istage_n; ++k)
        if (ix->istage_queued[k]) {
            cudaEventRecord(ix->ev_istage_used[k], s);
            ix->istage_queued[k] = false;
        }
    return st;
}

void drop_insertions(dbl_index *ix)
{
    ix->edges_stored -= ix->pending_edges;
    ix->pending.clear();
    ix->pending_edges = 0;
    for (int k = 0; k < dbl_index::kMaxIStage; ++k) ix->istage_queued[k] = false;
}

static unsigned blocks_for(int64_t work, int64_t cap_mult = 16)
{
    int64_t bl = (work + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)num_sms() * cap_mult;
    if (bl > cap) bl = cap;
    if (bl < 1) bl = 1;
    return (unsigned)bl;
}

dbl_status insert_edges(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, cudaStream_t s)
{
    if (b == 0) return DBL_OK;
    if (ix->edges_stored + b > ix->edge_cap)
        return fail(ix, DBL_ERR_CAPACITY, "insert: edge capacity exhausted (dbl_options.edge_capacity)");
    if (deferring(ix)) {
        if (ix->pending_edges + b >= (1ll << 31))
            if (dbl_status st = flush_insertions(ix, s)) return st;
        // the scratch of the whole queue is sized now; queued batches have not
        // used the old one yet, so it may be replaced
        if (dbl_status st = ensure_ins_scratch(ix, ix->pending_edges + b, s)) return st;
        ix->pending.push_back(dbl_index::Pending{src, dst, b});
        ix->pending_edges += b;
        ix->edges_stored += b;
        atomic_add_host_stat(ix, 15, (uint64_t)b, s);
        if ((int)ix->pending.size() == kMaxGroup) return flush_insertions(ix, s);
        return DBL_OK;
    }
    if (dbl_status st = ensure_ins_scratch(ix, b, s)) return st;
    return insert_edges_core(ix, src, dst, b, ix->ins_pos, ix->ins_pos + ix->ins_bcap, s);
}

// The insertion itself, with the per-edge scratch (2 x b int32: each edge's
// rank in its source's and its destination's batch) supplied by the caller.
dbl_status insert_edges_core(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, int32_t *pos_out,
                             int32_t *pos_in, cudaStream_t s)
{
    if (b == 0) return DBL_OK;
    if (ix->edges_stored + b > ix->edge_cap)
        return fail(ix, DBL_ERR_CAPACITY, "insert: edge capacity exhausted (dbl_options.edge_capacity)");
    if (ix->opt.flags & DBL_FLAG_PERSISTENT) return insert_persistent(ix, src, dst, b, pos_out, pos_in, s);
    const int32_t n = ix->n;
    const unsigned grid = blocks_for(b);
    // 1. validate before anything changes
    tbegin(ix, DBL_KERNEL_INSERT_APPEND, s);
    k_ins_validate<<<grid, kBlock, 0, s>>>(src, dst, b, n, ix->d_status);
    ++ix->launches;
    tend(ix, s);
    // The synchronous form reports a bad id before anything else runs; the
    // asynchronous persistent form leaves it latched (every mutating kernel
    // below then does nothing) and dbl_sync reports it.
    const bool no_sync = (ix->opt.flags & DBL_FLAG_ASYNC) && (ix->opt.flags & DBL_FLAG_PERSISTENT);
    if (!no_sync) {
        dbl_status st = read_status(ix, s);
        if (st) return fail(ix, st, "insert: vertex id out of range");
    }
    // 2. append
    int32_t *cnt_out = ix->ins_cnt, *cnt_in = ix->ins_cnt + ix->n_cap;  // [2][n_cap], zero between calls
    tbegin(ix, DBL_KERNEL_INSERT_APPEND, s);
    k_ins_count<<<grid, kBlock, 0, s>>>(src, dst, b, cnt_out, cnt_in, pos_out, pos_in, ix->d_stats, ix->d_status,
                                        dev_graph(ix).dirty);
    ++ix->launches;
    k_ins_grow<<<grid, kBlock, 0, s>>>(src, dst, b, cnt_out, cnt_in, pos_out, pos_in, ix->vm, ix->pool_out,
                                       ix->pool_in, ix->d_pool_top, ix->pool_cap, ix->d_status);
    ++ix->launches;
    k_ins_write<<<grid, kBlock, 0, s>>>(src, dst, b, pos_out, pos_in, ix->vm, ix->pool_out, ix->pool_in,
                                        ix->d_status);
    ++ix->launches;
    k_ins_commit<<<grid, kBlock, 0, s>>>(src, dst, b, cnt_out, cnt_in, pos_out, pos_in, ix->vm, ix->d_status);
    ++ix->launches;
    ix->edges_stored += b;
    atomic_add_host_stat(ix, 15, (uint64_t)b, s);
    // 3. seed the repair frontier, then propagate to the fixpoint
    FrontierOut f{ix->front[0], ix->d_counts + kCntFront0, ix->front_cap, mark_of(ix, 0), ix->wpd, ix->d_status};
    cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
    const DevGraph g = dev_graph(ix);
    tbegin(ix, DBL_KERNEL_INSERT_SEED, s);
    const uint64_t dlm = ix->dl_mask;
    switch (ix->packed ? 0 : ix->hs * 16 + ix->wd) {
    case 0: k_ins_seed<1, 0><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 2 * 16 + 1: k_ins_seed<2, 1><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 4 * 16 + 1: k_ins_seed<4, 1><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 4 * 16 + 2: k_ins_seed<4, 2><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 8 * 16 + 1: k_ins_seed<8, 1><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 8 * 16 + 2: k_ins_seed<8, 2><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    case 8 * 16 + 4: k_ins_seed<8, 4><<<grid, kBlock, 0, s>>>(src, dst, b, g, ix->rec, dlm, f, ix->d_stats); ++ix->launches; break;
    default: return fail(ix, DBL_ERR_INVALID, "insert: unsupported label width");
    }
    tend(ix, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "insert kernels");
    return propagate(ix, s);
}

}  // namespace dbl
