// Frontier helpers shared by label build, insertion repair and propagation.
//
// A frontier is a list of tasks (vertex, chunk, direction); a vertex whose
// edge list in that direction has d edges contributes ceil(d / kChunk) tasks,
// so a hub of degree 10^5 is spread over many teams instead of one.
//
// Vertices are deduplicated per level by a bitmap per direction (n bits,
// L2-resident: 0.6 MB per direction at 4.8M vertices).  Two bitmaps
// alternate: the frontier of level L is marked in bitmap L%2, and level L
// clears its own vertices' bits as it consumes them (the task of chunk 0), so
// every bitmap is empty again when a propagation reaches its fixpoint and no
// state carries over between propagations (or CUDA graph replays).
#pragma once

#include "dbl_internal.cuh"

namespace dbl {

struct FrontierOut {
    FTask *tasks;
    uint32_t *count;
    int64_t cap;
    uint32_t *mark;  // dedup bitmap of the frontier being filled: [2 directions][wpd words]
    int64_t wpd;     // words per direction
    uint32_t *status;
};

// Try to mark x in direction dir; true if this call set the bit.  A vertex
// with no edges in that direction has nothing to push: its bit is given back
// (so it stays clear for later levels) and the call returns false.
__device__ __forceinline__ bool mark_new(const FrontierOut &f, int dir, int32_t x, int32_t deg)
{
    uint32_t *w = f.mark + (size_t)dir * (size_t)f.wpd + (x >> 5);
    const uint32_t bit = 1u << (x & 31);
    const uint32_t old = atomicOr(w, bit);  // independent of deg: both loads are in flight together
    if (old & bit) return false;
    if (deg > 0) return true;
    atomicAnd(w, ~bit);
    return false;
}

// Clear x's bit in the bitmap its frontier was marked in (by the consumer of
// x's chunk-0 task).
__device__ __forceinline__ void mark_clear(uint32_t *mark, int64_t wpd, int dir, int32_t x)
{
    atomicAnd(mark + (size_t)dir * (size_t)wpd + (x >> 5), ~(1u << (x & 31)));
}

// Warp-cooperative enqueue: every lane of the warp must call it (lanes with
// want == false pass through).  One atomicAdd per warp reserves the slots.
__device__ __forceinline__ void warp_enqueue(bool want, int32_t x, int dir, const DevGraph &g,
                                             const FrontierOut &f)
{
    const int lane = threadIdx.x & 31;
    uint32_t nchunks = 0;
    AdjRange r{0, 0, 0, 0};
    if (want) {
        r = adj_of(g, dir, x);
        const int32_t d = r.bd + r.od;
        if (mark_new(f, dir, x, d)) nchunks = (uint32_t)((d + kChunk - 1) / kChunk);
    }
    uint32_t incl = nchunks;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(f.count, total);
    base = __shfl_sync(kFull, base, 31);
    uint32_t pos = base + incl - nchunks;
    for (uint32_t c = 0; c < nchunks; ++c, ++pos) {
        if ((int64_t)pos < f.cap) store_ftask(f.tasks, pos, make_ftask(x, dir, (int32_t)c, r));
        else set_status(f.status, DBL_ERR_CAPACITY);
    }
}

// Block-staged form of warp_enqueue.  Warps reserve room in a shared-memory
// stage with a shared-memory CAS; stage_flush (every thread of the block)
// then reserves the block's whole stage in the global frontier with one
// atomicAdd, so a level costs one global reservation per block instead of one
// per warp and iteration (all of them on the same word).  A warp whose tasks
// do not fit in the stage reserves global slots itself.
constexpr uint32_t kStage = 1024;  // 16 KB of tasks per block

struct Stage {
    FTask *tasks;  // shared, kStage entries
    uint32_t *n;   // shared, entries used
};

// Reserve room for `cnt` items per lane (warp-collective): in the block's
// stage if they fit, else straight in the global frontier.  Returns the
// lane's first position and whether it is global.
__device__ __forceinline__ uint32_t stage_reserve(uint32_t cnt, const FrontierOut &f, const Stage &st, bool &global_out)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    global_out = false;
    if (total == 0) return 0;
    uint32_t base = 0, global = 0;
    if (lane == 31) {
        uint32_t old = *(volatile uint32_t *)st.n;
        for (;;) {  // ends: each failed CAS means another warp's reservation succeeded
            if (old + total > kStage) {
                global = 1;
                break;
            }
            const uint32_t prev = atomicCAS(st.n, old, old + total);
            if (prev == old) break;
            old = prev;
        }
        base = global ? atomicAdd(f.count, total) : old;
    }
    base = __shfl_sync(kFull, base, 31);
    global_out = __shfl_sync(kFull, global, 31) != 0;
    return base + incl - cnt;
}

__device__ __forceinline__ void stage_write(bool global, uint32_t pos, const FTask &t, const FrontierOut &f,
                                            const Stage &st)
{
    if (!global) st.tasks[pos] = t;
    else if ((int64_t)pos < f.cap) store_ftask(f.tasks, pos, t);
    else set_status(f.status, DBL_ERR_CAPACITY);
}

// The chunks of x (already marked) into the stage; warp-collective.
__device__ __forceinline__ void stage_put(uint32_t nchunks, int32_t x, int dir, const AdjRange &r,
                                          const FrontierOut &f, const Stage &st)
{
    bool global;
    uint32_t pos = stage_reserve(nchunks, f, st, global);
    for (uint32_t c = 0; c < nchunks; ++c, ++pos) stage_write(global, pos, make_ftask(x, dir, (int32_t)c, r), f, st);
}

// One ready task per lane (has) into the stage; warp-collective.
__device__ __forceinline__ void stage_put_task(bool has, const FTask &t, const FrontierOut &f, const Stage &st)
{
    bool global;
    const uint32_t pos = stage_reserve(has ? 1u : 0u, f, st, global);
    if (has) stage_write(global, pos, t, f, st);
}

// Mark x in the frontier being filled and, if it is new there, stage its
// chunks; warp-collective (lanes with want == false pass through).
// stage_enqueue with x's adjacency already loaded (r is read only if want).
__device__ __forceinline__ void stage_enqueue_at(bool want, int32_t x, int dir, const AdjRange &r,
                                                 const FrontierOut &f, const Stage &st)
{
    uint32_t nchunks = 0;
    if (want) {
        const int32_t d = r.bd + r.od;
        if (mark_new(f, dir, x, d)) nchunks = (uint32_t)((d + kChunk - 1) / kChunk);
    }
    stage_put(nchunks, x, dir, r, f, st);
}

__device__ __forceinline__ void stage_enqueue(bool want, int32_t x, int dir, const DevGraph &g, const FrontierOut &f,
                                              const Stage &st)
{
    stage_enqueue_at(want, x, dir, want ? adj_of(g, dir, x) : AdjRange{0, 0, 0, 0}, f, st);
}

// Move the block's stage to the global frontier; every thread of the block
// calls it.  Leaves the stage empty.
__device__ __forceinline__ void stage_flush(const FrontierOut &f, const Stage &st)
{
    __shared__ uint32_t s_base;
    __syncthreads();
    const uint32_t cnt = *(volatile uint32_t *)st.n;
    if (threadIdx.x == 0 && cnt) s_base = atomicAdd(f.count, cnt);
    __syncthreads();
    if (cnt) {
        const uint32_t b = s_base;
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t pos = b + i;
            if ((int64_t)pos < f.cap) store_ftask(f.tasks, pos, st.tasks[i]);
            else set_status(f.status, DBL_ERR_CAPACITY);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *st.n = 0;
    __syncthreads();
}

// Declares this block's stage (shared memory) and empties it; every thread calls it.
#define DBL_BLOCK_STAGE(name)                                                                                         \
    __shared__ ::dbl::FTask name##_tasks[::dbl::kStage];                                                              \
    __shared__ uint32_t name##_n;                                                                                     \
    if (threadIdx.x == 0) name##_n = 0;                                                                               \
    __syncthreads();                                                                                                  \
    const ::dbl::Stage name{name##_tasks, &name##_n}

// Shared-memory append buffer of int32 items for one block: a push from any
// lane (divergent code included) is a shared-memory atomic; istage_flush (every
// thread of the block) moves the items to a global list with one reservation
// per block.  Items that do not fit are appended to the global list directly.
constexpr uint32_t kIStage = 2048;

struct IStage {
    int32_t *items;  // shared, kIStage entries
    uint32_t *n;     // shared, pushes so far (may exceed kIStage)
};

struct IList {
    int32_t *items;
    uint32_t *count;
    int64_t cap;
    uint32_t *overflow;  // set when the list is full (may be null: cannot overflow)
};

__device__ __forceinline__ void istage_push(const IStage &st, int32_t item, const IList &dst)
{
    const uint32_t pos = atomicAdd(st.n, 1u);
    if (pos < kIStage) {
        st.items[pos] = item;
        return;
    }
    const uint32_t g = atomicAdd(dst.count, 1u);
    if ((int64_t)g < dst.cap) dst.items[g] = item;
    else if (dst.overflow) atomicExch(dst.overflow, 1u);
}

__device__ __forceinline__ void istage_flush(const IStage &st, const IList &dst)
{
    __shared__ uint32_t s_base;
    __syncthreads();
    uint32_t cnt = *(volatile uint32_t *)st.n;
    if (cnt > kIStage) cnt = kIStage;
    if (threadIdx.x == 0 && cnt) s_base = atomicAdd(dst.count, cnt);
    __syncthreads();
    if (cnt) {
        const uint32_t b = s_base;
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t pos = b + i;
            if ((int64_t)pos < dst.cap) dst.items[pos] = st.items[i];
            else if (dst.overflow) atomicExch(dst.overflow, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *st.n = 0;
    __syncthreads();
}

#define DBL_BLOCK_ISTAGE(name)                                                                                        \
    __shared__ int32_t name##_items[::dbl::kIStage];                                                                  \
    __shared__ uint32_t name##_n;                                                                                     \
    if (threadIdx.x == 0) name##_n = 0;                                                                               \
    __syncthreads();                                                                                                  \
    const ::dbl::IStage name{name##_items, &name##_n}

// Block-uniform reservation: every thread of the block calls it with its own
// count and gets the start of its own range; the block's total is reserved in
// *gcount with one atomicAdd.  *total receives the block's total.
__device__ __forceinline__ uint32_t block_reserve(uint32_t mine, uint32_t *gcount, uint32_t *total)
{
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_base, s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const uint32_t t = s_w[w];
            s_w[w] = run;
            run += t;
        }
        s_total = run;
        s_base = run ? atomicAdd(gcount, run) : 0u;
    }
    __syncthreads();
    const uint32_t r = s_base + s_w[warp] + incl - mine;
    *total = s_total;
    __syncthreads();
    return r;
}

// Same, for callers whose loop is not warp-uniform: uses the active mask.
__device__ __forceinline__ void any_enqueue(int32_t x, int dir, const DevGraph &g, const FrontierOut &f)
{
    const AdjRange r = adj_of(g, dir, x);
    const int32_t d = r.bd + r.od;
    if (!mark_new(f, dir, x, d)) return;
    const uint32_t nchunks = (uint32_t)((d + kChunk - 1) / kChunk);
    uint32_t pos = atomicAdd(f.count, nchunks);
    for (uint32_t c = 0; c < nchunks; ++c, ++pos) {
        if ((int64_t)pos < f.cap) store_ftask(f.tasks, pos, make_ftask(x, dir, (int32_t)c, r));
        else set_status(f.status, DBL_ERR_CAPACITY);
    }
}

}  // namespace dbl
