// Batched reachability queries (Algorithm 2).
//
// Label test, one thread per pair, in Algorithm 2's order:
//   u == v                                  -> true   (Des(u) contains u, Table 1)
//   DL_out(u) & DL_in(v)  != 0              -> true   (Lemma 1)
//   BL_in(u) not within BL_in(v), or
//   BL_out(v) not within BL_out(u)          -> false  (Lemma 2)
//   DL_out(v) & DL_in(u)  != 0              -> false  (Theorem 1)
//   DL_out(u) & DL_in(u) or same for v      -> false  (Theorem 2)
//   otherwise undecided: compacted for the pruned search.
//
// Pruned search: the undecided pairs are grouped 64 to a word; group g's
// search state at vertex x is one slot of a device hash table keyed by
// (g, x): `visit` holds the queries whose search has reached x and `pend` the
// ones to expand from x at the next level.  A task expands (x, g, mask) over
// up to kChunk out-edges; for each edge x -> y and each query j in the mask:
// y == v_j marks j found; otherwise j is pruned at y if DL_out(u_j) meets
// DL_in(y) or y fails BL_Contain(y, v_j) (Algorithm 2's two prunes, in its
// order); the rest are OR-ed into y's visit bits, and bits new there are
// pending for the next level.  All groups of a batch run in one wave; if the
// table or task list overflows, the wave's found answers are kept and the
// groups are rerun in halves.
#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_kernels.cuh"

namespace dbl {

__host__ __device__ constexpr int hs_of(int words) { return words <= 2 ? 2 : (words <= 4 ? 4 : 8); }

// ------------------------------------------------------------ label test
template <int WD, int WB>
__global__ void __launch_bounds__(kBlock) k_query_label(const int32_t *qu, const int32_t *qv, int64_t q,
                                                        const uint64_t *rec, int32_t n, uint8_t *ans,
                                                        uint8_t *code, int32_t *und, uint32_t *n_und,
                                                        uint32_t *status, unsigned long long *stats)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    __shared__ unsigned int cnt[8];
    if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < q; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool undecided = false;
        if (i < q) {
            const int32_t u = __ldcs(qu + i), v = __ldcs(qv + i);
            uint8_t a = 0, c = DBL_CODE_UNDECIDED;
            if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
                set_status(status, DBL_ERR_INVALID);
            } else if (u == v) {
                a = 1;
                c = DBL_CODE_SELF;
            } else {
                uint64_t fu[HS], bu[HS], fv[HS], bv[HS];
                load_half<HS>(rec + (size_t)u * RW, fu);
                load_half<HS>(rec + (size_t)u * RW + HS, bu);
                load_half<HS>(rec + (size_t)v * RW, fv);
                load_half<HS>(rec + (size_t)v * RW + HS, bv);
                uint64_t uv = 0, vu = 0, uu = 0, vv = 0, blf = 0;
#pragma unroll
                for (int w = 0; w < WD; ++w) {
                    uv |= bu[w] & fv[w];
                    vu |= bv[w] & fu[w];
                    uu |= bu[w] & fu[w];
                    vv |= bv[w] & fv[w];
                }
#pragma unroll
                for (int w = WD; w < WD + WB; ++w) blf |= (fu[w] & ~fv[w]) | (bv[w] & ~bu[w]);
                if (uv) {
                    a = 1;
                    c = DBL_CODE_DL;
                } else if (blf) {
                    c = DBL_CODE_BL;
                } else if (vu) {
                    c = DBL_CODE_THM1;
                } else if (uu | vv) {
                    c = DBL_CODE_THM2;
                } else {
                    undecided = true;
                }
            }
            __stcs(ans + i, a);
            if (code) __stcs(code + i, c);
            if (c) atomicAdd(&cnt[c], 1u);
        }
        const unsigned bal = __ballot_sync(kFull, undecided);
        if (bal) {
            uint32_t b0 = 0;
            const int leader = __ffs(bal) - 1;
            if (lane == leader) b0 = atomicAdd(n_und, (uint32_t)__popc(bal));
            b0 = __shfl_sync(kFull, b0, leader);
            if (undecided) und[b0 + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
    __syncthreads();
    if (threadIdx.x < 8 && cnt[threadIdx.x]) atomicAdd(stats + threadIdx.x, (unsigned long long)cnt[threadIdx.x]);
}

// ------------------------------------------------------------ search
__device__ __forceinline__ unsigned long long mix_key(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct SearchCtx {
    SearchSlot *table;
    unsigned long long slot_mask;
    int32_t *claimed;
    uint32_t *n_claimed;
    uint32_t *overflow;
};

constexpr int kMaxProbe = 2048;

__device__ __forceinline__ int64_t slot_find_or_insert(const SearchCtx &c, unsigned long long key)
{
    unsigned long long h = mix_key(key) & c.slot_mask;
    for (int p = 0; p < kMaxProbe; ++p) {
        SearchSlot *s = c.table + h;
        unsigned long long k = __ldcg(&s->key);
        if (k == key) return (int64_t)h;
        if (k == kEmptyKey) {
            unsigned long long prev = atomicCAS(&s->key, kEmptyKey, key);
            if (prev == kEmptyKey) {
                uint32_t pos = atomicAdd(c.n_claimed, 1u);
                c.claimed[pos] = (int32_t)h;  // pos < slots: each slot is claimed once
                return (int64_t)h;
            }
            if (prev == key) return (int64_t)h;
        }
        h = (h + 1) & c.slot_mask;
    }
    atomicExch(c.overflow, 1u);
    return -1;
}

// qtab word layout per query: [u | v<<32][DL_out(u) x WD][BL_in(v) x WB][BL_out(v) x WB]
template <int WD, int WB>
struct QT {
    static constexpr int W = 1 + WD + 2 * WB;
};

struct SlotList {
    int32_t *items;
    uint32_t *count;
    int64_t cap;
};

__device__ __forceinline__ void mark_pending(const SearchCtx &c, int64_t slot, unsigned long long bits,
                                             uint32_t epoch, const SlotList &next)
{
    SearchSlot *s = c.table + slot;
    atomicOr(&s->pend, bits);
    if (atomicExch(&s->stamp, epoch) != epoch) {
        uint32_t pos = atomicAdd(next.count, 1u);
        if ((int64_t)pos < next.cap) next.items[pos] = (int32_t)slot;
        else atomicExch(c.overflow, 1u);
    }
}

// Wave setup: queries [j0, j1) of the undecided list (groups j/64).
template <int WD, int WB>
__global__ void k_search_setup(const int32_t *und, int64_t j0, int64_t j1, const int32_t *qu, const int32_t *qv,
                               const uint64_t *rec, uint64_t *qtab, SearchCtx c, uint32_t epoch, SlotList first)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = und[j];
        const int32_t u = qu[i], v = qv[i];
        uint64_t *t = qtab + (size_t)j * W;
        t[0] = (uint64_t)(uint32_t)u | ((uint64_t)(uint32_t)v << 32);
        const uint64_t *ru = rec + (size_t)u * RW, *rv = rec + (size_t)v * RW;
#pragma unroll
        for (int w = 0; w < WD; ++w) t[1 + w] = ru[HS + w];              // DL_out(u)
#pragma unroll
        for (int w = 0; w < WB; ++w) {
            t[1 + WD + w] = rv[WD + w];                                   // BL_in(v)
            t[1 + WD + WB + w] = rv[HS + WD + w];                         // BL_out(v)
        }
        const unsigned long long g = (unsigned long long)(j >> 6);
        const unsigned long long bit = 1ull << (j & 63);
        int64_t s = slot_find_or_insert(c, (g << 32) | (uint32_t)u);
        if (s < 0) continue;
        atomicOr(&c.table[s].visit, bit);
        mark_pending(c, s, bit, epoch, first);
    }
}

// Slots listed for the next level -> tasks (x, g, chunk, mask) over Suc(x).
__global__ void k_search_finalize(const SlotList cur, DevGraph g, SearchCtx c, SearchTask *tasks,
                                  uint32_t *n_tasks, int64_t task_cap)
{
    const uint32_t n = *cur.count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n && i < cur.cap;
         i += (int64_t)gridDim.x * blockDim.x) {
        SearchSlot *s = c.table + cur.items[i];
        const unsigned long long mask = atomicExch(&s->pend, 0ull);
        if (!mask) continue;
        const unsigned long long key = s->key;
        const int32_t x = (int32_t)(uint32_t)key;
        const int32_t d = deg_of(g, 0, x);
        const uint32_t nch = (uint32_t)((d + kChunk - 1) / kChunk);
        if (!nch) continue;
        uint32_t pos = atomicAdd(n_tasks, nch);
        for (uint32_t ch = 0; ch < nch; ++ch, ++pos) {
            if ((int64_t)pos >= task_cap) {
                atomicExch(c.overflow, 1u);
                break;
            }
            SearchTask t;
            t.x = x;
            t.g = (uint32_t)(key >> 32);
            t.chunk = ch;
            t.pad = 0;
            t.mask = mask;
            tasks[pos] = t;
        }
    }
}

template <int WD, int WB, int TEAM>
__global__ void __launch_bounds__(kBlock) k_search_expand(const SearchTask *tasks, const uint32_t *n_tasks_p,
                                                          int64_t task_cap, DevGraph g, const uint64_t *rec,
                                                          const uint64_t *qtab, unsigned long long *found,
                                                          SearchCtx c, uint32_t epoch, SlotList next,
                                                          unsigned long long *stats)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    constexpr int TPW = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int team = lane / TEAM, tl = lane % TEAM;
    int64_t ntasks = *n_tasks_p;
    if (ntasks > task_cap) ntasks = task_cap;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long relaxed = 0;
    for (int64_t wb = warp0 * TPW; wb < ntasks; wb += nwarps * TPW) {
        const int64_t t = wb + team;
        if (t >= ntasks) continue;
        const SearchTask tk = tasks[t];
        const unsigned long long fg = __ldcg(found + tk.g);
        const unsigned long long m = tk.mask & ~fg;
        if (!m) continue;
        const AdjRange r = adj_of(g, 0, tk.x);
        const int32_t d = r.bd + r.od;
        const int32_t lo = (int32_t)tk.chunk * kChunk;
        const int32_t hi = min(d, lo + kChunk);
        const uint64_t *qg = qtab + (size_t)tk.g * 64 * W;
        for (int32_t e = lo + tl; e < hi; e += TEAM) {
            const int32_t y = adj_at(g, 0, r, e);
            ++relaxed;
            uint64_t fy[HS], by[HS];
            load_half<HS>(rec + (size_t)y * RW, fy);       // DL_in(y) | BL_in(y)
            load_half<HS>(rec + (size_t)y * RW + HS, by);  // DL_out(y) | BL_out(y)
            unsigned long long hits = 0, allowed = 0, rest = m;
            while (rest) {
                const int b = __ffsll((long long)rest) - 1;
                rest &= rest - 1;
                const uint64_t *qj = qg + (size_t)b * W;
                const uint64_t uv = __ldg(qj);
                const unsigned long long bit = 1ull << b;
                if ((int32_t)(uint32_t)(uv >> 32) == y) {
                    hits |= bit;
                    continue;
                }
                uint64_t dl = 0, bl = 0;
#pragma unroll
                for (int w = 0; w < WD; ++w) dl |= __ldg(qj + 1 + w) & fy[w];
                if (dl) continue;
#pragma unroll
                for (int w = 0; w < WB; ++w)
                    bl |= (fy[WD + w] & ~__ldg(qj + 1 + WD + w)) | (__ldg(qj + 1 + WD + WB + w) & ~by[WD + w]);
                if (bl) continue;
                allowed |= bit;
            }
            if (hits) atomicOr(found + tk.g, hits);
            if (allowed) {
                const int64_t s = slot_find_or_insert(c, ((unsigned long long)tk.g << 32) | (uint32_t)y);
                if (s < 0) continue;
                const unsigned long long old = atomicOr(&c.table[s].visit, allowed);
                const unsigned long long nb = allowed & ~old;
                if (nb) mark_pending(c, s, nb, epoch, next);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) relaxed += __shfl_xor_sync(kFull, relaxed, o);
    if (lane == 0 && relaxed) atomicAdd(stats + 10, relaxed);
}

__global__ void k_search_answer(const int32_t *und, int64_t j0, int64_t j1, const unsigned long long *found,
                                int final_wave, uint8_t *ans, uint8_t *code, unsigned long long *stats)
{
    __shared__ unsigned int cnt[2];
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1;
         j += (int64_t)gridDim.x * blockDim.x) {
        const bool hit = (found[j >> 6] >> (j & 63)) & 1ull;
        const int64_t i = und[j];
        if (hit) {
            ans[i] = 1;
            if (code) code[i] = DBL_CODE_BFS_POS;
            atomicAdd(&cnt[0], 1u);
        } else if (final_wave) {
            ans[i] = 0;
            if (code) code[i] = DBL_CODE_BFS_NEG;
            atomicAdd(&cnt[1], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt[0]) atomicAdd(stats + DBL_CODE_BFS_POS, (unsigned long long)cnt[0]);
        if (cnt[1]) atomicAdd(stats + DBL_CODE_BFS_NEG, (unsigned long long)cnt[1]);
    }
}

__global__ void k_search_clear(SearchSlot *table, const int32_t *claimed, const uint32_t *n_claimed)
{
    const uint32_t n = *n_claimed;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        SearchSlot *s = table + claimed[i];
        s->key = kEmptyKey;
        s->visit = 0;
        s->pend = 0;
        s->stamp = 0;
    }
}

// ------------------------------------------------------------ host driver
static unsigned blocks_for(int64_t work)
{
    int64_t b = (work + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)num_sms() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <int WD, int WB>
static dbl_status run_search_wave(dbl_index *ix, const int32_t *qu, const int32_t *qv, int64_t j0, int64_t j1,
                                  uint8_t *ans, uint8_t *code, bool *overflowed, cudaStream_t s)
{
    uint32_t *cnt = ix->d_counts;
    uint32_t *h = ix->h_pinned;
    SearchCtx c{ix->table, (unsigned long long)(ix->table_slots - 1), ix->claimed, cnt + kCntClaimed,
                cnt + kCntOverflow};
    const int64_t g0 = j0 >> 6, g1 = (j1 + 63) >> 6;
    cudaMemsetAsync(ix->found + g0, 0, sizeof(unsigned long long) * (size_t)(g1 - g0), s);
    cudaMemsetAsync(cnt + kCntSlots0, 0, sizeof(uint32_t) * 5, s);  // slots0, slots1, tasks, claimed, overflow
    ix->epoch += 1;
    SlotList lists[2] = {{ix->slot_list[0], cnt + kCntSlots0, ix->table_slots},
                         {ix->slot_list[1], cnt + kCntSlots1, ix->table_slots}};
    tbegin(ix, DBL_KERNEL_SEARCH_OTHER, s);
    k_search_setup<WD, WB><<<blocks_for(j1 - j0), kBlock, 0, s>>>(ix->und, j0, j1, qu, qv, ix->rec, ix->qtab, c,
                                                                   ix->epoch, lists[0]);
    ++ix->launches;
    tend(ix, s);
    int cur = 0;
    int64_t levels = 0;
    const int64_t max_levels = (int64_t)ix->n + 2;
    for (;;) {
        cudaMemcpyAsync(h, cnt, sizeof(uint32_t) * kCntWords, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(ix, e, "search level");
        if (h[kCntOverflow]) break;
        const uint32_t nslots = h[kCntSlots0 + cur];
        if (!nslots) break;
        if (++levels > max_levels) {
            ix->poisoned = true;
            return fail(ix, DBL_ERR_TIMEOUT, "search: level bound exceeded");
        }
        const int nxt = cur ^ 1;
        cudaMemsetAsync(cnt + kCntTasks, 0, sizeof(uint32_t), s);
        cudaMemsetAsync(cnt + kCntSlots0 + nxt, 0, sizeof(uint32_t), s);
        tbegin(ix, DBL_KERNEL_SEARCH_OTHER, s);
        k_search_finalize<<<blocks_for(nslots), kBlock, 0, s>>>(lists[cur], dev_graph(ix), c, ix->stask,
                                                                 cnt + kCntTasks, ix->stask_cap);
        ++ix->launches;
        tbegin(ix, DBL_KERNEL_SEARCH_EXPAND, s);
        ix->epoch += 1;
        // tasks are at most nslots * (1 + maxdeg/kChunk); size the grid generously and let it stride
        const int64_t est = (int64_t)nslots * 2;
        switch (ix->opt.team) {
        case 4:
            k_search_expand<WD, WB, 4><<<blocks_for(est * 4), kBlock, 0, s>>>(
                ix->stask, cnt + kCntTasks, ix->stask_cap, dev_graph(ix), ix->rec, ix->qtab, ix->found, c, ix->epoch,
                lists[nxt], ix->d_stats);
            ++ix->launches;
            break;
        case 16:
            k_search_expand<WD, WB, 16><<<blocks_for(est * 16), kBlock, 0, s>>>(
                ix->stask, cnt + kCntTasks, ix->stask_cap, dev_graph(ix), ix->rec, ix->qtab, ix->found, c, ix->epoch,
                lists[nxt], ix->d_stats);
            ++ix->launches;
            break;
        default:
            k_search_expand<WD, WB, 8><<<blocks_for(est * 8), kBlock, 0, s>>>(
                ix->stask, cnt + kCntTasks, ix->stask_cap, dev_graph(ix), ix->rec, ix->qtab, ix->found, c, ix->epoch,
                lists[nxt], ix->d_stats);
            ++ix->launches;
            break;
        }
        tend(ix, s);
        cur = nxt;
    }
    *overflowed = h[kCntOverflow] != 0;
    tbegin(ix, DBL_KERNEL_SEARCH_OTHER, s);
    k_search_answer<<<blocks_for(j1 - j0), kBlock, 0, s>>>(ix->und, j0, j1, ix->found, *overflowed ? 0 : 1, ans, code,
                                                            ix->d_stats);
    ++ix->launches;
    k_search_clear<<<blocks_for(ix->table_slots / 4), kBlock, 0, s>>>(ix->table, ix->claimed, cnt + kCntClaimed);
    ++ix->launches;
    tend(ix, s);
    atomic_add_host_stat(ix, 14, 1, s);
    atomic_add_host_stat(ix, 8, (uint64_t)levels, s);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(ix, e, "search wave") : DBL_OK;
}

template <int WD, int WB>
static dbl_status query_t(dbl_index *ix, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans, uint8_t *code,
                          cudaStream_t s)
{
    dbl_status st = ensure_search_scratch(ix, q, s);
    if (st) return st;
    uint32_t *cnt = ix->d_counts;
    cudaMemsetAsync(cnt + kCntUnd, 0, sizeof(uint32_t), s);
    int64_t blocks = (q + kBlock - 1) / kBlock;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    tbegin(ix, DBL_KERNEL_QUERY_LABEL, s);
    k_query_label<WD, WB><<<(unsigned)blocks, kBlock, 0, s>>>(u, v, q, ix->rec, ix->n, ans, code, ix->und,
                                                              cnt + kCntUnd, ix->d_status, ix->d_stats);
    ++ix->launches;
    tend(ix, s);
    uint32_t *h = ix->h_pinned;
    cudaMemcpyAsync(h, cnt + kCntUnd, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h + 8, ix->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(ix, e, "query label test");
    if (h[8]) {
        cudaMemsetAsync(ix->d_status, 0, sizeof(uint32_t), s);  // consumed; nothing was changed
        return fail(ix, (dbl_status)h[8], "query: vertex id out of range");
    }
    const int64_t U = h[0];
    if (!U) return DBL_OK;
    // waves: all groups at once; on overflow rerun the unanswered in halves
    struct Range {
        int64_t j0, j1;
    };
    std::vector<Range> stack{{0, U}};
    while (!stack.empty()) {
        Range r = stack.back();
        stack.pop_back();
        bool over = false;
        st = run_search_wave<WD, WB>(ix, u, v, r.j0, r.j1, ans, code, &over, s);
        if (st) return st;
        if (over) {
            const int64_t groups = (r.j1 - r.j0 + 63) / 64;
            if (groups <= 1) return fail(ix, DBL_ERR_CAPACITY, "search: one group overflowed the state table");
            const int64_t mid = r.j0 + (groups / 2) * 64;
            stack.push_back({mid, r.j1});
            stack.push_back({r.j0, mid});
        }
    }
    return DBL_OK;
}

dbl_status query(dbl_index *ix, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans, uint8_t *code,
                 cudaStream_t s)
{
    if (q == 0) return DBL_OK;
    const int key = ix->wd * 16 + ix->wb;
    switch (key) {
    case 1 * 16 + 1: return query_t<1, 1>(ix, u, v, q, ans, code, s);
    case 2 * 16 + 1: return query_t<2, 1>(ix, u, v, q, ans, code, s);
    case 1 * 16 + 2: return query_t<1, 2>(ix, u, v, q, ans, code, s);
    case 2 * 16 + 2: return query_t<2, 2>(ix, u, v, q, ans, code, s);
    case 4 * 16 + 1: return query_t<4, 1>(ix, u, v, q, ans, code, s);
    case 1 * 16 + 4: return query_t<1, 4>(ix, u, v, q, ans, code, s);
    case 2 * 16 + 4: return query_t<2, 4>(ix, u, v, q, ans, code, s);
    case 4 * 16 + 2: return query_t<4, 2>(ix, u, v, q, ans, code, s);
    case 4 * 16 + 4: return query_t<4, 4>(ix, u, v, q, ans, code, s);
    default: return fail(ix, DBL_ERR_INVALID, "unsupported (k, kprime) combination");
    }
}

}  // namespace dbl
