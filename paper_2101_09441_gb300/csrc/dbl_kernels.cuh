// Device bodies shared by the per-level kernels and the persistent kernels.
#pragma once

#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"

namespace dbl {

__device__ __forceinline__ void warp_stat_add(unsigned long long *stats, int idx, unsigned long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(stats + idx, v);
}

// Owner lane of flat position e, given each lane's exclusive prefix `excl`
// (non-decreasing over lanes, excl of lane 0 = 0): the largest lane k with
// excl_k <= e.  Every lane of the warp must call it.
__device__ __forceinline__ int flat_owner(uint32_t excl, uint32_t e)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
        const uint32_t v = __shfl_sync(kFull, excl, lo + step);
        if (v <= e) lo += step;
    }
    return lo;
}

// Local continuation: a vertex that a warp's pushes change, and whose edges
// fit in one task, goes to the warp's own list (shared memory) instead of the
// next level's frontier, and the warp processes its list in further rounds of
// the same level (up to kLocalRounds), so chains of small vertices advance
// several hops per grid barrier.  The vertex is marked in the next level's
// bitmap as usual; the warp clears the bit before it reads the vertex's
// record, with a fence in between: a push that lands after the read then finds
// the bit clear and enqueues the vertex again (its atomicOr has returned
// before it marks), so no bit is lost.  What is left in a list after the last
// local round goes to the next level.
constexpr int kLocal = 32;
constexpr int kLocalRounds = 8;

// A changed neighbour x joins the next level (or the warp's local list) in
// two halves, so that the memory operations of several edges (x's adjacency
// metadata, its bit in the next level's bitmap) can be in flight together
// before the warp-collective half runs: local_mark returns the number of x's
// chunks when this call marked x (0 otherwise) ...
__device__ __forceinline__ uint32_t local_mark(bool want, int32_t x, int dir, const DevGraph &g,
                                               const FrontierOut &f, AdjRange &r)
{
    r = AdjRange{0, 0, 0, 0};
    if (!want) return 0;
    r = adj_of(g, dir, x);
    const int32_t d = r.bd + r.od;
    return mark_new(f, dir, x, d) ? (uint32_t)((d + kChunk - 1) / kChunk) : 0u;
}

// ... and local_put places the marked vertices (warp-collective).
__device__ __forceinline__ void local_put(uint32_t nchunks, int32_t x, int dir, const AdjRange &r,
                                          const FrontierOut &f, const Stage &st, FTask *wl, int &wl_n)
{
    const int lane = threadIdx.x & 31;
    const bool loc = nchunks == 1;
    const unsigned bl = __ballot_sync(kFull, loc);
    const int rank = __popc(bl & ((1u << lane) - 1u));
    const bool to_local = loc && wl_n + rank < kLocal;
    if (to_local) wl[wl_n + rank] = make_ftask(x, dir, 0, r);
    wl_n = min(kLocal, wl_n + __popc(bl));
    stage_put(to_local ? 0u : nchunks, x, dir, r, f, st);
}

// One round of the flattened level: lane-held tasks (has, tk); their
// vertices' bits are cleared in clear_mark (fence after the clear when the
// bitmap is the one being filled: local tasks).  The warp takes U x 32 edges
// per step, and the column loads, then the neighbours' half-records, then
// the ORs, then the marks of a step are issued together (U edges of each lane
// in flight at each stage).
template <int HS, int U>
__device__ __forceinline__ void flat_round(const DevGraph &g, const RecView &rw, bool has, const FTask &tk,
                                           uint32_t *clear_mark, bool local, const FrontierOut &f, const Stage &st,
                                           FTask *wl, int &wl_n, unsigned long long &relaxed,
                                           unsigned long long &ntask)
{
    const int lane = threadIdx.x & 31;
    int32_t col0 = 0, ncol = 0, pool0 = 0;
    uint32_t cnt = 0;
    int dir = 0;
    uint64_t rv[HS];
#pragma unroll
    for (int i = 0; i < HS; ++i) rv[i] = 0;
    if (has) {
        dir = task_dir(tk);
        if (task_first(tk)) {
            mark_clear(clear_mark, f.wpd, dir, tk.v);
            if (local) __threadfence();
        }
        col0 = tk.col0;
        ncol = task_ncol(tk);
        pool0 = tk.pool0;
        cnt = (uint32_t)task_edges(tk);
        load_half<HS>(rec_half(rw, tk.v, dir), rv);
        ++ntask;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t base = 0; base < total; base += 32u * U) {
        int odir[U];
        int32_t x[U];
        bool ok[U], want[U];
        uint64_t orv[U][HS], rx[U][HS];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint32_t e = base + 32u * k + lane;
            const int owner = flat_owner(excl, e);
            odir[k] = __shfl_sync(kFull, dir, owner);
            const int32_t ocol0 = __shfl_sync(kFull, col0, owner), oncol = __shfl_sync(kFull, ncol, owner);
            const int32_t opool0 = __shfl_sync(kFull, pool0, owner);
            const int32_t oe = (int32_t)(e - __shfl_sync(kFull, excl, owner));
#pragma unroll
            for (int i = 0; i < HS; ++i) orv[k][i] = __shfl_sync(kFull, rv[i], owner);
            ok[k] = e < total;
            x[k] = ok[k] ? task_edge(g, odir[k], ocol0, oncol, opool0, oe) : 0;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (ok[k]) load_half<HS>(rec_half(rw, x[k], odir[k]), rx[k]);
            else {
#pragma unroll
                for (int i = 0; i < HS; ++i) rx[k][i] = ~0ull;  // nothing to add
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            want[k] = false;
            relaxed += ok[k] ? 1 : 0;
            uint64_t *px = rec_half(rw, x[k], odir[k]);
#pragma unroll
            for (int i = 0; i < HS; ++i) {
                if (orv[k][i] & ~rx[k][i]) {
                    const unsigned long long old = atomicOr((unsigned long long *)(px + i), orv[k][i]);
                    want[k] |= (orv[k][i] & ~old) != 0;
                }
            }
            if (want[k]) mark_dirty(g.dirty, x[k]);
        }
        uint32_t nch[U];
        AdjRange r[U];
#pragma unroll
        for (int k = 0; k < U; ++k) nch[k] = local_mark(want[k], x[k], odir[k], g, f, r[k]);
#pragma unroll
        for (int k = 0; k < U; ++k) local_put(nch[k], x[k], odir[k], r[k], f, st, wl, wl_n);
    }
}

// Flattened level (TEAM == 1): each lane takes one task per round (task
// w + nwarps*(32r + lane) for warp w, so a hub's consecutive chunks land in
// different warps), and the warp walks the concatenation of its tasks' edges
// 32 at a time; each edge's task data come from the owner lane by shuffles.
// A round costs ceil(edges of the warp's tasks / 32) iterations, whatever the
// mix of task sizes.  Then the warp's local rounds (above).
template <int HS, int U>
__device__ __forceinline__ void expand_level_flat(const DevGraph &g, const RecView &rw, const FTask *tasks,
                                                  uint32_t ntasks, uint32_t *cur_mark, const FrontierOut &f,
                                                  unsigned long long *stats, int64_t warp, int64_t nwarps,
                                                  const Stage &st)
{
    __shared__ FTask s_wl[32 * kLocal];
    const int lane = threadIdx.x & 31;
    FTask *wl = s_wl + (threadIdx.x >> 5) * kLocal;
    int wl_n = 0;  // warp-uniform
    unsigned long long relaxed = 0, ntask = 0;
    if ((int64_t)ntasks > f.cap) ntasks = (uint32_t)f.cap;  // both frontier buffers have the same capacity
    for (int64_t r0 = 0; warp + nwarps * r0 < (int64_t)ntasks; r0 += 32) {  // warp-uniform
        const int64_t t = warp + nwarps * (r0 + lane);
        const bool has = t < (int64_t)ntasks;
        const FTask tk = has ? load_ftask(tasks, t) : FTask{0, 0u, 0, 0};
        flat_round<HS, U>(g, rw, has, tk, cur_mark, false, f, st, wl, wl_n, relaxed, ntask);
    }
    for (int lr = 0; lr < kLocalRounds && wl_n > 0; ++lr) {
        __syncwarp();
        const bool has = lane < wl_n;
        const FTask tk = has ? wl[lane] : FTask{0, 0u, 0, 0};
        __syncwarp();
        wl_n = 0;
        flat_round<HS, U>(g, rw, has, tk, f.mark, true, f, st, wl, wl_n, relaxed, ntask);
    }
    __syncwarp();
    {
        const bool has = lane < wl_n;  // left for the next level (already marked there)
        const FTask tk = has ? wl[lane] : FTask{0, 0u, 0, 0};
        stage_put_task(has, tk, f, st);
    }
    warp_stat_add(stats, 9, ntask);
    warp_stat_add(stats, 10, relaxed);
    stage_flush(f, st);
}

// One level of label propagation over `ntasks` tasks, processed by warps
// [warp0, warp0 + nwarps*k) in steps of nwarps.  Every lane of a warp runs the
// same number of iterations (warp_enqueue needs the whole warp).  The tasks'
// vertices are cleared from cur_mark, the bitmap their frontier was marked in.
//
// New tasks go through the block's stage (stage_enqueue); the stage is flushed
// at the end, so every thread of the block must call this.
template <int HS, int TEAM, int U = 1>
__device__ __forceinline__ void expand_level(const DevGraph &g, const RecView &rw, const FTask *tasks,
                                             uint32_t ntasks, uint32_t *cur_mark, const FrontierOut &f,
                                             unsigned long long *stats, int64_t warp0, int64_t nwarps,
                                             const Stage &st)
{
    if constexpr (TEAM == 1) {
        expand_level_flat<HS, U>(g, rw, tasks, ntasks, cur_mark, f, stats, warp0, nwarps, st);
    } else {
        constexpr int TPW = 32 / TEAM;
        const int lane = threadIdx.x & 31;
        const int team = lane / TEAM, tl = lane % TEAM;
        unsigned long long relaxed = 0, ntask = 0;
        if ((int64_t)ntasks > f.cap) ntasks = (uint32_t)f.cap;  // both frontier buffers have the same capacity
        for (int64_t wb = warp0 * TPW; wb < (int64_t)ntasks; wb += nwarps * TPW) {
            const int64_t t = wb + team;
            const bool has = t < (int64_t)ntasks;
            int32_t col0 = 0, ncol = 0, pool0 = 0, cnt = 0;
            int dir = 0;
            uint64_t rv[HS];
#pragma unroll
            for (int i = 0; i < HS; ++i) rv[i] = 0;
            if (has) {
                const FTask tk = load_ftask(tasks, t);
                dir = task_dir(tk);
                if (task_first(tk) && tl == 0) mark_clear(cur_mark, f.wpd, dir, tk.v);
                col0 = tk.col0;
                ncol = task_ncol(tk);
                pool0 = tk.pool0;
                cnt = task_edges(tk);
                load_half<HS>(rec_half(rw, tk.v, dir), rv);
                if (tl == 0) ++ntask;
            }
            int iters = (cnt + TEAM - 1) / TEAM;
#pragma unroll
            for (int o = 16; o; o >>= 1) iters = max(iters, __shfl_xor_sync(kFull, iters, o));
            for (int it = 0; it < iters; ++it) {
                const int32_t e = it * TEAM + tl;
                bool want = false;
                int32_t x = 0;
                if (has && e < cnt) {
                    x = task_edge(g, dir, col0, ncol, pool0, e);
                    ++relaxed;
                    uint64_t *px = rec_half(rw, x, dir);
                    uint64_t rx[HS];
                    load_half<HS>(px, rx);
                    bool changed = false;
#pragma unroll
                    for (int i = 0; i < HS; ++i) {
                        if (rv[i] & ~rx[i]) {
                            unsigned long long old = atomicOr((unsigned long long *)(px + i), rv[i]);
                            changed |= (rv[i] & ~old) != 0;
                        }
                    }
                    want = changed;
                    if (changed) mark_dirty(g.dirty, x);
                }
                stage_enqueue(want, x, dir, g, f, st);
            }
        }
        warp_stat_add(stats, 9, ntask);
        warp_stat_add(stats, 10, relaxed);
        stage_flush(f, st);
    }
}

}  // namespace dbl
