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

namespace dbl {

template <int HS, int TEAM>
__global__ void __launch_bounds__(kBlock) k_expand(DevGraph g, uint64_t *rec, const uint64_t *tasks,
                                                   const uint32_t *ntasks_p, FrontierOut f,
                                                   unsigned long long *stats)
{
    expand_level<HS, TEAM>(g, rec, tasks, *ntasks_p, f, stats,
                           ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           ((int64_t)gridDim.x * blockDim.x) >> 5);
}

template <int HS, int TEAM>
static void launch_expand(dbl_index *ix, int cur, uint32_t ntasks, const FrontierOut &f, cudaStream_t s)
{
    constexpr int TPW = 32 / TEAM;
    int64_t warps = ((int64_t)ntasks + TPW - 1) / TPW;
    int64_t blocks = (warps * 32 + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_expand<HS, TEAM><<<(unsigned)blocks, kBlock, 0, s>>>(dev_graph(ix), ix->rec, ix->front[cur],
                                                           ix->d_counts + kCntFront0 + cur, f, ix->d_stats);
    ++ix->launches;
}

template <int HS>
static void launch_expand_team(dbl_index *ix, int cur, uint32_t ntasks, const FrontierOut &f, cudaStream_t s)
{
    switch (ix->opt.team) {
    case 4: launch_expand<HS, 4>(ix, cur, ntasks, f, s); break;
    case 16: launch_expand<HS, 16>(ix, cur, ntasks, f, s); break;
    case 32: launch_expand<HS, 32>(ix, cur, ntasks, f, s); break;
    default: launch_expand<HS, 8>(ix, cur, ntasks, f, s); break;
    }
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
        ix->epoch += 1;
        const int nxt = cur ^ 1;
        FrontierOut f{ix->front[nxt], ix->d_counts + kCntFront0 + nxt, ix->front_cap, ix->stamp, ix->epoch,
                      ix->d_status};
        cudaMemsetAsync(ix->d_counts + kCntFront0 + nxt, 0, sizeof(uint32_t), s);
        tbegin(ix, DBL_KERNEL_PROPAGATE, s);
        switch (ix->hs) {
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

dbl_status propagate_persistent(dbl_index *ix, cudaStream_t s)
{
    const int32_t flags = ix->opt.flags;
    ix->opt.flags &= ~DBL_FLAG_PERSISTENT;
    dbl_status st = propagate(ix, s);
    ix->opt.flags = flags;
    return st;
}

}  // namespace dbl
