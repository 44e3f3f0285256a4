// Label propagation to the least fixpoint.
//
// Build (Algorithm 1) runs one BFS per landmark and per leaf bucket; insertion
// repair (Algorithm 3 and its mirrors, Section 5) runs a pruned BFS per edge
// that ORs the source's label into every descendant until the label is already
// contained.  Both compute the least fixpoint of
//     fwd(x) = seed_f(x) | OR_{p in Pre(x)} fwd(p)      (DL_in | BL_in)
//     bwd(x) = seed_b(x) | OR_{s in Suc(x)} bwd(s)      (DL_out | BL_out)
// from a starting point below it, so here all k + k' bits of a half-record
// travel together: a task (x, chunk, dir) pushes x's half over up to kChunk
// of its edges, ORs it into each neighbour whose half is missing bits, and
// enqueues every neighbour that changed.  A neighbour that already contains
// the pushed bits is pruned, exactly Algorithm 3's test.  Level-synchronous;
// the fixpoint is reached when a level changes nothing.
#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_kernels.cuh"
#include "dbl_persistent.cuh"

namespace dbl {

// edges per lane in flight at each stage of a flattened level (team width 1)
constexpr int kPropUnroll = 2;

template <int HS, int TEAM>
__global__ void __launch_bounds__(kBlock) k_expand(DevGraph g, RecView rw, const FTask *tasks,
                                                   const uint32_t *ntasks_p, uint32_t *cur_mark, FrontierOut f,
                                                   unsigned long long *stats)
{
    DBL_BLOCK_STAGE(st);
    expand_level<HS, TEAM, kPropUnroll>(g, rw, tasks, *ntasks_p, cur_mark, f, stats,
                           ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           ((int64_t)gridDim.x * blockDim.x) >> 5, st);
}

template <int HS, int TEAM>
static void launch_expand(dbl_index *ix, int cur, uint32_t ntasks, const FrontierOut &f, cudaStream_t s)
{
    // tasks per warp at a time; the flattened form (TEAM 1) spreads about 8
    // tasks over each warp so that a hub's chunks land in different warps
    constexpr int TPW = TEAM == 1 ? 8 : 32 / TEAM;
    int64_t warps = ((int64_t)ntasks + TPW - 1) / TPW;
    int64_t blocks = (warps * 32 + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_expand<HS, TEAM><<<(unsigned)blocks, kBlock, 0, s>>>(prop_graph(ix), rec_view(ix), ix->front[cur],
                                                           ix->d_counts + kCntFront0 + cur, mark_of(ix, cur), f,
                                                           ix->d_stats);
    ++ix->launches;
}

template <int HS>
static void launch_expand_team(dbl_index *ix, int cur, uint32_t ntasks, const FrontierOut &f, cudaStream_t s)
{
    switch (ix->opt.team) {
    case 1: launch_expand<HS, 1>(ix, cur, ntasks, f, s); break;
    case 4: launch_expand<HS, 4>(ix, cur, ntasks, f, s); break;
    case 16: launch_expand<HS, 16>(ix, cur, ntasks, f, s); break;
    case 32: launch_expand<HS, 32>(ix, cur, ntasks, f, s); break;
    default: launch_expand<HS, 8>(ix, cur, ntasks, f, s); break;
    }
}

// Propagate over another record array with half width hs (used by the
// coverage pass of the learned scorer): the frontier kernels read the
// records and their width from the index, so swap them in for the call.
dbl_status propagate_records(dbl_index *ix, uint64_t *rec, int32_t hs, cudaStream_t s)
{
    uint64_t *rec0 = ix->rec;
    const int32_t hs0 = ix->hs, rw0 = ix->rw;
    ix->rec = rec;
    ix->hs = hs;
    ix->rw = 2 * hs;
    dbl_status st = propagate(ix, s);
    ix->rec = rec0;
    ix->hs = hs0;
    ix->rw = rw0;
    return st;
}

// A device error during propagation (a frontier overflow, which the sizing
// rules out) leaves labels short of the fixpoint: poison the index.
static dbl_status propagate_error(dbl_index *ix, uint32_t code, cudaStream_t s)
{
    cudaMemsetAsync(ix->d_status, 0, sizeof(uint32_t), s);
    ix->poisoned = true;
    return fail(ix, (dbl_status)code, "propagate: device error; index poisoned until dbl_restore");
}

dbl_status propagate(dbl_index *ix, cudaStream_t s)
{
    if (ix->opt.flags & DBL_FLAG_PERSISTENT) return propagate_persistent(ix, s);
    int cur = 0;
    uint32_t *h = ix->h_pinned;
    cudaMemcpyAsync(h, ix->d_counts, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h + 8, ix->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "propagate: sync");
    uint32_t ntasks = h[cur];
    int64_t levels = 0;
    const int64_t max_levels = (int64_t)ix->n + 2;
    while (ntasks > 0) {
        if (h[8]) return propagate_error(ix, h[8], s);
        if (++levels > max_levels) {
            ix->poisoned = true;
            return fail(ix, DBL_ERR_TIMEOUT, "propagate: level bound exceeded");
        }
        const int nxt = cur ^ 1;
        // frontier buffer i is marked in bitmap parity i
        FrontierOut f{ix->front[nxt], ix->d_counts + kCntFront0 + nxt, ix->front_cap, mark_of(ix, nxt), ix->wpd,
                      ix->d_status};
        cudaMemsetAsync(ix->d_counts + kCntFront0 + nxt, 0, sizeof(uint32_t), s);
        tbegin(ix, DBL_KERNEL_PROPAGATE, s);
        switch (ix->hs) {
        case 1: launch_expand_team<1>(ix, cur, ntasks, f, s); break;
        case 2: launch_expand_team<2>(ix, cur, ntasks, f, s); break;
        case 4: launch_expand_team<4>(ix, cur, ntasks, f, s); break;
        default: launch_expand_team<8>(ix, cur, ntasks, f, s); break;
        }
        tend(ix, s);
        cudaMemcpyAsync(h, ix->d_counts, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h + 8, ix->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(ix, e, "propagate: level");
        cur = nxt;
        ntasks = h[cur];
    }
    if (h[8]) return propagate_error(ix, h[8], s);
    // the fixpoint leaves frontier 0 as the (empty) starting buffer for the next call
    if (cur != 0) {
        cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
    }
    atomic_add_host_stat(ix, 8, (uint64_t)levels, s);
    return DBL_OK;
}


// ---------------------------------------------------------------------------
// Persistent form: one cooperative launch runs every level.  Level L reads
// frontier buffer L%2 with count c[L%3] and fills buffer (L+1)%2 / c[(L+1)%3];
// block 0 zeroes c[(L+2)%3], which nobody touches during level L.  One grid
// barrier per level; every block sees the same counts after it, so all take
// the same exit.  The level bound and the barrier's bounded wait turn any
// runaway into DBL_ERR_TIMEOUT instead of a hang.
template <int HS, int TEAM>
__global__ void __launch_bounds__(pblock_of(HS), 1)
    k_propagate_persistent(DevGraph g, RecView rw, FTask *f0, FTask *f1, uint32_t *c3, int64_t cap,
                           uint32_t *mark, int64_t wpd, uint32_t *status, unsigned long long *stats,
                           GridBarrier bar, int64_t max_levels)
{
    GridSync gs(bar);
    DBL_BLOCK_STAGE(st);
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t L = 0;
    for (;; ++L) {
        const uint32_t nt = ld_volatile_u32(c3 + L % 3);
        if (nt == 0 || ld_volatile_u32(status)) break;
        if (L >= max_levels) {
            set_status(status, DBL_ERR_TIMEOUT);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) c3[(L + 2) % 3] = 0;
        uint32_t *cur_mark = mark + (size_t)(L & 1) * 2 * (size_t)wpd;
        uint32_t *nxt_mark = mark + (size_t)((L + 1) & 1) * 2 * (size_t)wpd;
        FrontierOut f{(L & 1) ? f0 : f1, c3 + (L + 1) % 3, cap, nxt_mark, wpd, status};
        expand_level<HS, TEAM, kPropUnroll>(g, rw, (L & 1) ? f1 : f0, nt, cur_mark, f, stats, warp0, nwarps, st);
        if (!gs.sync(status)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[8] += (unsigned long long)L;
        c3[L % 3] = 0;
    }
    gs.leave();
}

template <int HS, int TEAM>
static dbl_status launch_persistent(dbl_index *ix, cudaStream_t s)
{
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_propagate_persistent<HS, TEAM>, pblock_of(HS), 0);
    if (blocks_per_sm < 1) return fail(ix, DBL_ERR_CUDA, "persistent propagate: kernel does not fit on an SM");
    DevGraph g = prop_graph(ix);
    FTask *f0 = ix->front[0], *f1 = ix->front[1];
    uint32_t *c3 = ix->d_counts + kCntP0;
    int64_t cap = ix->front_cap;
    uint32_t *mark = ix->mark;
    int64_t wpd = ix->wpd;
    uint32_t *status = ix->d_status;
    unsigned long long *stats = ix->d_stats;
    GridBarrier bar = grid_barrier_at(ix->d_counts);
    if (ix->opt.flags & DBL_FLAG_TIMING) bar.trace = ix->d_trace;
    int64_t max_levels = (int64_t)ix->n + 2;
    RecView rw = rec_view(ix);
    void *args[] = {&g, &rw, &f0, &f1, &c3, &cap, &mark, &wpd, &status, &stats, &bar, &max_levels};
    dim3 grid((unsigned)num_sms()), block(pblock_of(HS));
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_propagate_persistent<HS, TEAM>, grid, block, args, 0, s);
    ++ix->launches;
    return e ? cuda_fail(ix, e, "persistent propagate launch") : DBL_OK;
}

template <int HS>
static dbl_status launch_persistent_team(dbl_index *ix, cudaStream_t s)
{
    switch (ix->opt.team) {
    case 1: return launch_persistent<HS, 1>(ix, s);
    case 4: return launch_persistent<HS, 4>(ix, s);
    case 16: return launch_persistent<HS, 16>(ix, s);
    case 32: return launch_persistent<HS, 32>(ix, s);
    default: return launch_persistent<HS, 8>(ix, s);
    }
}

dbl_status propagate_persistent(dbl_index *ix, cudaStream_t s)
{
    // the starting frontier is buffer 0 with its count in kCntFront0
    cudaMemcpyAsync(ix->d_counts + kCntP0, ix->d_counts + kCntFront0, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(ix->d_counts + kCntP0 + 1, 0, 2 * sizeof(uint32_t), s);
    tbegin(ix, DBL_KERNEL_PROPAGATE, s);
    dbl_status st;
    switch (ix->hs) {
    case 1: st = launch_persistent_team<1>(ix, s); break;
    case 2: st = launch_persistent_team<2>(ix, s); break;
    case 4: st = launch_persistent_team<4>(ix, s); break;
    default: st = launch_persistent_team<8>(ix, s); break;
    }
    tend(ix, s);
    cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
    if (st) return st;
    if (ix->opt.flags & DBL_FLAG_ASYNC) return DBL_OK;  // errors surface through dbl_sync
    uint32_t code = 0;
    cudaMemcpyAsync(ix->h_pinned + 8, ix->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "persistent propagate");
    code = ix->h_pinned[8];
    return code ? propagate_error(ix, code, s) : DBL_OK;
}

// ---------------------------------------------------------------------------
// Check of the bounded grid barrier (dbl_barrier_probe): every block but
// `absent` meets at one barrier of the index's barrier words, whose wait
// gives up after bar.spin_limit polls; the absent block only leaves.  With
// absent < 0 every block arrives and the launch ends without error; otherwise
// the waits run out, DBL_ERR_TIMEOUT is latched, and every block still leaves
// (the last one resets the barrier words for the next launch).
__global__ void k_barrier_probe(GridBarrier bar, uint32_t *status, int absent)
{
    GridSync gs(bar);
    if ((int)blockIdx.x != absent) gs.sync(status);
    gs.leave();
}

dbl_status barrier_probe(dbl_index *ix, int64_t spin_limit, int32_t absent, cudaStream_t s)
{
    GridBarrier bar = grid_barrier_at(ix->d_counts);
    bar.spin_limit = (unsigned long long)spin_limit;
    uint32_t *status = ix->d_status;
    int ab = absent;
    void *args[] = {&bar, &status, &ab};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3((unsigned)num_sms()), dim3(32),
                                                args, 0, s);
    ++ix->launches;
    return e ? cuda_fail(ix, e, "barrier probe launch") : DBL_OK;
}

}  // namespace dbl
