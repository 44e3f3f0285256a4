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
#include "dbl_persistent.cuh"

namespace dbl {

__host__ __device__ constexpr int hs_of(int words) { return words <= 2 ? 2 : (words <= 4 ? 4 : 8); }

// ------------------------------------------------------------ label test
// Each thread takes QPT queries (QPT = 4 for 32-byte records) and issues all
// of their record loads before using any, so that many DRAM sectors are in
// flight per warp; answers and codes are written coalesced, the deciding
// rules are counted with warp ballots, and undecided pairs are compacted with
// one atomic per warp.
template <int WD, int WB, int QPT>
__global__ void __launch_bounds__(kBlock) k_query_label(const int32_t *qu, const int32_t *qv, int64_t q,
                                                        const uint64_t *rec, int32_t n, uint8_t *ans,
                                                        uint8_t *code, int32_t *und, uint32_t *n_und,
                                                        uint32_t *status, unsigned long long *stats)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    const int lane = threadIdx.x & 31;
    unsigned int counts[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // kept by lane 0
    const int64_t tile = (int64_t)blockDim.x * QPT;
    const int64_t stride = (int64_t)gridDim.x * tile;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < q; base += stride) {
        int32_t u[QPT], v[QPT];
        bool live[QPT];
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
            live[j] = i < q;
            u[j] = live[j] ? __ldcs(qu + i) : 0;
            v[j] = live[j] ? __ldcs(qv + i) : 0;
        }
        bool ok[QPT];
        uint64_t fu[QPT][HS], bu[QPT][HS], fv[QPT][HS], bv[QPT][HS];
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            ok[j] = live[j] && (uint32_t)u[j] < (uint32_t)n && (uint32_t)v[j] < (uint32_t)n && u[j] != v[j];
            const int32_t uu = ok[j] ? u[j] : 0, vv = ok[j] ? v[j] : 0;
            load_half<HS>(rec + (size_t)uu * RW, fu[j]);
            load_half<HS>(rec + (size_t)uu * RW + HS, bu[j]);
            load_half<HS>(rec + (size_t)vv * RW, fv[j]);
            load_half<HS>(rec + (size_t)vv * RW + HS, bv[j]);
        }
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
            uint8_t a = 0, c = DBL_CODE_UNDECIDED;
            bool undecided = false;
            if (live[j]) {
                if ((uint32_t)u[j] >= (uint32_t)n || (uint32_t)v[j] >= (uint32_t)n) {
                    set_status(status, DBL_ERR_INVALID);
                } else if (u[j] == v[j]) {
                    a = 1;
                    c = DBL_CODE_SELF;
                } else {
                    uint64_t uv = 0, vu = 0, su = 0, sv = 0, blf = 0;
#pragma unroll
                    for (int w = 0; w < WD; ++w) {
                        uv |= bu[j][w] & fv[j][w];
                        vu |= bv[j][w] & fu[j][w];
                        su |= bu[j][w] & fu[j][w];
                        sv |= bv[j][w] & fv[j][w];
                    }
#pragma unroll
                    for (int w = WD; w < WD + WB; ++w) blf |= (fu[j][w] & ~fv[j][w]) | (bv[j][w] & ~bu[j][w]);
                    if (uv) {
                        a = 1;
                        c = DBL_CODE_DL;
                    } else if (blf) {
                        c = DBL_CODE_BL;
                    } else if (vu) {
                        c = DBL_CODE_THM1;
                    } else if (su | sv) {
                        c = DBL_CODE_THM2;
                    } else {
                        undecided = true;
                    }
                }
                __stcs(ans + i, a);
                if (code) __stcs(code + i, c);
            }
#pragma unroll
            for (int r = 1; r < 6; ++r) counts[r] += __popc(__ballot_sync(kFull, live[j] && c == r));
            const unsigned bal = __ballot_sync(kFull, undecided);
            if (bal) {
                uint32_t b0 = 0;
                const int leader = __ffs(bal) - 1;
                if (lane == leader) b0 = atomicAdd(n_und, (uint32_t)__popc(bal));
                b0 = __shfl_sync(kFull, b0, leader);
                if (undecided) und[b0 + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
            }
        }
    }
    if (lane == 0)
#pragma unroll
        for (int r = 1; r < 6; ++r)
            if (counts[r]) atomicAdd(stats + r, (unsigned long long)counts[r]);
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

struct SlotList {
    int32_t *items;
    uint32_t *count;
    int64_t cap;
};

// Everything a search phase needs (both forms).
struct SearchArgs {
    DevGraph g;
    const uint64_t *rec;
    uint64_t *qtab;
    unsigned long long *found;
    SearchCtx c;
    SearchTask *tasks;
    int64_t task_cap;
    const int32_t *und;
    const int32_t *qu, *qv;
    uint8_t *ans, *code;
    unsigned long long *stats;
    int32_t *lists[2];
    int64_t list_cap;
};

// Device-side state of the persistent search.
struct PersistState {
    uint32_t list_count[2];
    uint32_t task_count[2];
    uint32_t n_claimed;
    uint32_t overflow;
    int32_t top;
    int32_t pad;
    long long range[2];
    long long stack[64][2];
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
                c.claimed[pos] = (int32_t)h;  // pos < slots: each slot is claimed once per wave
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

// Wave setup: queries [j0, j1) of the undecided list (group j/64, bit j%64):
// fill the query table, zero the groups' found words, and start every search
// at its u (visited and pending there).
template <int WD, int WB>
__device__ __forceinline__ void search_setup(const SearchArgs &a, int64_t j0, int64_t j1, uint32_t epoch,
                                             const SlotList &first)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gq = (j0 >> 6) + t0; gq < ((j1 + 63) >> 6); gq += nt) a.found[gq] = 0;
    for (int64_t j = j0 + t0; j < j1; j += nt) {
        const int64_t i = a.und[j];
        const int32_t u = a.qu[i], v = a.qv[i];
        uint64_t *t = a.qtab + (size_t)j * W;
        t[0] = (uint64_t)(uint32_t)u | ((uint64_t)(uint32_t)v << 32);
        const uint64_t *ru = a.rec + (size_t)u * RW, *rv = a.rec + (size_t)v * RW;
#pragma unroll
        for (int w = 0; w < WD; ++w) t[1 + w] = ru[HS + w];              // DL_out(u)
#pragma unroll
        for (int w = 0; w < WB; ++w) {
            t[1 + WD + w] = rv[WD + w];                                   // BL_in(v)
            t[1 + WD + WB + w] = rv[HS + WD + w];                         // BL_out(v)
        }
        const unsigned long long g = (unsigned long long)(j >> 6);
        const unsigned long long bit = 1ull << (j & 63);
        int64_t s = slot_find_or_insert(a.c, (g << 32) | (uint32_t)u);
        if (s < 0) continue;
        atomicOr(&a.c.table[s].visit, bit);
        mark_pending(a.c, s, bit, epoch, first);
    }
}

// Slots listed for the next level -> tasks (x, g, chunk, mask) over Suc(x);
// one task-list reservation per warp.
__device__ __forceinline__ void search_finalize(const SearchArgs &a, const SlotList &cur, uint32_t *n_tasks)
{
    const int64_t n = min((int64_t)ld_volatile_u32(cur.count), cur.cap);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        unsigned long long mask = 0, key = 0;
        uint32_t nch = 0;
        int32_t x = 0;
        if (i < n) {
            SearchSlot *s = a.c.table + cur.items[i];
            mask = atomicExch(&s->pend, 0ull);
            if (mask) {
                key = s->key;
                x = (int32_t)(uint32_t)key;
                nch = (uint32_t)((deg_of(a.g, 0, x) + kChunk - 1) / kChunk);
            }
        }
        uint32_t incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        uint32_t wbase = 0;
        if (lane == 31) wbase = atomicAdd(n_tasks, total);
        wbase = __shfl_sync(kFull, wbase, 31);
        uint32_t pos = wbase + incl - nch;
        for (uint32_t ch = 0; ch < nch; ++ch, ++pos) {
            if ((int64_t)pos >= a.task_cap) {
                atomicExch(a.c.overflow, 1u);
                break;
            }
            SearchTask t;
            t.x = x;
            t.g = (uint32_t)(key >> 32);
            t.chunk = ch;
            t.pad = 0;
            t.mask = mask;
            a.tasks[pos] = t;
        }
    }
}

// One search level: for each task's edges x -> y and each live query j of the
// task's mask, in Algorithm 2's order: y == v_j -> found; DL prune; BL prune;
// otherwise y is visited for j, and bits new at y are pending for next level.
template <int WD, int WB, int TEAM>
__device__ __forceinline__ void search_expand(const SearchArgs &a, uint32_t n_tasks_in, uint32_t epoch,
                                              const SlotList &next)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    constexpr int TPW = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int team = lane / TEAM, tl = lane % TEAM;
    const int64_t ntasks = min((int64_t)n_tasks_in, a.task_cap);
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long relaxed = 0;
    for (int64_t wb = warp0 * TPW; wb < ntasks; wb += nwarps * TPW) {
        const int64_t t = wb + team;
        if (t >= ntasks) continue;
        const SearchTask tk = a.tasks[t];
        const unsigned long long m = tk.mask & ~__ldcg(a.found + tk.g);
        if (!m) continue;
        const AdjRange r = adj_of(a.g, 0, tk.x);
        const int32_t d = r.bd + r.od;
        const int32_t lo = (int32_t)tk.chunk * kChunk;
        const int32_t hi = min(d, lo + kChunk);
        const uint64_t *qg = a.qtab + (size_t)tk.g * 64 * W;
        for (int32_t e = lo + tl; e < hi; e += TEAM) {
            const int32_t y = adj_at(a.g, 0, r, e);
            ++relaxed;
            uint64_t fy[HS], by[HS];
            load_half<HS>(a.rec + (size_t)y * RW, fy);       // DL_in(y) | BL_in(y)
            load_half<HS>(a.rec + (size_t)y * RW + HS, by);  // DL_out(y) | BL_out(y)
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
            if (hits) atomicOr(a.found + tk.g, hits);
            if (allowed) {
                const int64_t s = slot_find_or_insert(a.c, ((unsigned long long)tk.g << 32) | (uint32_t)y);
                if (s < 0) continue;
                const unsigned long long old = atomicOr(&a.c.table[s].visit, allowed);
                const unsigned long long nb = allowed & ~old;
                if (nb) mark_pending(a.c, s, nb, epoch, next);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) relaxed += __shfl_xor_sync(kFull, relaxed, o);
    if (lane == 0 && relaxed) atomicAdd(a.stats + 10, relaxed);
}

// Answers of queries [j0, j1): found -> true (bfs_pos); otherwise false
// (bfs_neg) when the wave ran to exhaustion (final), else left for a rerun.
__device__ __forceinline__ void search_answer(const SearchArgs &a, int64_t j0, int64_t j1, bool final_wave)
{
    __shared__ unsigned int cnt[2];
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1;
         j += (int64_t)gridDim.x * blockDim.x) {
        const bool hit = (__ldcg(a.found + (j >> 6)) >> (j & 63)) & 1ull;
        const int64_t i = a.und[j];
        if (hit) {
            a.ans[i] = 1;
            if (a.code) a.code[i] = DBL_CODE_BFS_POS;
            atomicAdd(&cnt[0], 1u);
        } else if (final_wave) {
            a.ans[i] = 0;
            if (a.code) a.code[i] = DBL_CODE_BFS_NEG;
            atomicAdd(&cnt[1], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt[0]) atomicAdd(a.stats + DBL_CODE_BFS_POS, (unsigned long long)cnt[0]);
        if (cnt[1]) atomicAdd(a.stats + DBL_CODE_BFS_NEG, (unsigned long long)cnt[1]);
    }
}

// Return every slot claimed in the wave to empty.
__device__ __forceinline__ void search_clear(const SearchArgs &a)
{
    const uint32_t n = ld_volatile_u32(a.c.n_claimed);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        SearchSlot *s = a.c.table + a.c.claimed[i];
        s->key = kEmptyKey;
        s->visit = 0;
        s->pend = 0;
        s->stamp = 0;
    }
}

// ------------------------------------------------------------ per-level kernels
template <int WD, int WB>
__global__ void k_search_setup(SearchArgs a, int64_t j0, int64_t j1, uint32_t epoch, SlotList first)
{
    search_setup<WD, WB>(a, j0, j1, epoch, first);
}

__global__ void k_search_finalize(SearchArgs a, SlotList cur, uint32_t *n_tasks) { search_finalize(a, cur, n_tasks); }

template <int WD, int WB, int TEAM>
__global__ void __launch_bounds__(kBlock) k_search_expand(SearchArgs a, const uint32_t *n_tasks, uint32_t epoch,
                                                          SlotList next)
{
    search_expand<WD, WB, TEAM>(a, ld_volatile_u32(n_tasks), epoch, next);
}

__global__ void k_search_answer(SearchArgs a, int64_t j0, int64_t j1, int final_wave)
{
    search_answer(a, j0, j1, final_wave != 0);
}

__global__ void k_search_clear(SearchArgs a) { search_clear(a); }

// ------------------------------------------------------------ persistent kernel
// All waves and levels of one query batch in one cooperative launch.  Block 0
// keeps a stack of query ranges (an overflowing wave is split in halves) and
// the phase counters; every decision is read by all blocks after a barrier.
// Per level: finalize, barrier, expand, barrier.
template <int WD, int WB, int TEAM>
__device__ __forceinline__ void search_waves(const SearchArgs &a, PersistState *ps, const uint32_t *n_und,
                                             GridSync &gs, uint32_t *status, int64_t max_levels)
{
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    const uint32_t U = ld_volatile_u32(n_und);
    if (U == 0) return;
    if (leader) {
        ps->top = 1;
        ps->stack[0][0] = 0;
        ps->stack[0][1] = U;
    }
    unsigned long long levels = 0, waves = 0;
    for (;;) {
        if (leader) {
            if (ps->top > 0) {
                --ps->top;
                ps->range[0] = ps->stack[ps->top][0];
                ps->range[1] = ps->stack[ps->top][1];
            } else {
                ps->range[0] = ps->range[1] = -1;
            }
            ps->list_count[0] = ps->list_count[1] = 0;
            ps->task_count[0] = ps->task_count[1] = 0;
            ps->n_claimed = 0;
            ps->overflow = 0;
        }
        if (!gs.sync(status)) return;
        const long long j0 = *(volatile long long *)&ps->range[0], j1 = *(volatile long long *)&ps->range[1];
        if (j0 < 0 || ld_volatile_u32(status)) break;
        ++waves;
        SlotList lists[2] = {{a.lists[0], &ps->list_count[0], a.list_cap}, {a.lists[1], &ps->list_count[1], a.list_cap}};
        uint32_t sep = 1;
        search_setup<WD, WB>(a, j0, j1, sep, lists[0]);
        if (!gs.sync(status)) return;
        for (int64_t L = 0;; ++L) {
            const int cur = (int)(L & 1);
            if (!ld_volatile_u32(&ps->list_count[cur]) || ld_volatile_u32(&ps->overflow) || ld_volatile_u32(status))
                break;
            if (L >= max_levels) {
                set_status(status, DBL_ERR_TIMEOUT);
                break;
            }
            ++levels;
            search_finalize(a, lists[cur], &ps->task_count[cur]);
            if (!gs.sync(status)) return;
            ++sep;
            if (leader) {
                ps->list_count[cur] = 0;
                ps->task_count[cur ^ 1] = 0;
            }
            search_expand<WD, WB, TEAM>(a, ld_volatile_u32(&ps->task_count[cur]), sep, lists[cur ^ 1]);
            if (!gs.sync(status)) return;
        }
        const bool over = ld_volatile_u32(&ps->overflow) != 0;
        search_answer(a, j0, j1, !over);
        search_clear(a);
        if (!gs.sync(status)) return;
        if (over && leader) {
            const long long groups = (j1 - j0 + 63) / 64;
            if (groups <= 1 || ps->top + 2 > 64) {
                set_status(status, DBL_ERR_CAPACITY);
            } else {
                const long long mid = j0 + (groups / 2) * 64;
                ps->stack[ps->top][0] = mid;
                ps->stack[ps->top][1] = j1;
                ps->stack[ps->top + 1][0] = j0;
                ps->stack[ps->top + 1][1] = mid;
                ps->top += 2;
            }
        }
    }
    if (leader) {
        a.stats[8] += levels;
        a.stats[14] += waves;
    }
}

template <int WD, int WB, int TEAM>
__global__ void __launch_bounds__(pblock_of(hs_of(WD + WB)), 1)
    k_search_persistent(SearchArgs a, PersistState *ps, const uint32_t *n_und, GridBarrier bar, uint32_t *status,
                        int64_t max_levels)
{
    GridSync gs(bar);
    search_waves<WD, WB, TEAM>(a, ps, n_und, gs, status, max_levels);
    gs.leave();
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

static SearchArgs search_args(dbl_index *ix, dbl_qctx *c, const int32_t *qu, const int32_t *qv, uint8_t *ans,
                              uint8_t *code, uint32_t *n_claimed, uint32_t *overflow)
{
    SearchArgs a;
    a.g = dev_graph(ix);
    a.rec = ix->rec;
    a.qtab = c->qtab;
    a.found = c->found;
    a.c = SearchCtx{c->table, (unsigned long long)(c->table_slots - 1), c->claimed, n_claimed, overflow};
    a.tasks = c->stask;
    a.task_cap = c->stask_cap;
    a.und = c->und;
    a.qu = qu;
    a.qv = qv;
    a.ans = ans;
    a.code = code;
    a.stats = ix->d_stats;
    a.lists[0] = c->slot_list[0];
    a.lists[1] = c->slot_list[1];
    a.list_cap = c->table_slots;
    return a;
}

// Kernel timing brackets are kept for the index's own context only (they are
// not thread-safe; explicit contexts may run on several host threads).
static void qt_begin(dbl_index *ix, dbl_qctx *c, int kind, cudaStream_t s)
{
    if (c == ix->qc) tbegin(ix, kind, s);
}
static void qt_end(dbl_index *ix, dbl_qctx *c, cudaStream_t s)
{
    if (c == ix->qc) tend(ix, s);
}

template <int WD, int WB>
static void launch_search_expand(dbl_index *ix, dbl_qctx *c, const SearchArgs &a, int64_t est, uint32_t sep,
                                 const SlotList &next, cudaStream_t s)
{
    uint32_t *nt = c->d_counts + kCntTasks;
    switch (ix->opt.team) {
    case 4: k_search_expand<WD, WB, 4><<<blocks_for(est * 4), kBlock, 0, s>>>(a, nt, sep, next); break;
    case 16:
    case 32: k_search_expand<WD, WB, 16><<<blocks_for(est * 16), kBlock, 0, s>>>(a, nt, sep, next); break;
    default: k_search_expand<WD, WB, 8><<<blocks_for(est * 8), kBlock, 0, s>>>(a, nt, sep, next); break;
    }
    ++ix->launches;
}

template <int WD, int WB>
static dbl_status run_search_wave(dbl_index *ix, dbl_qctx *c, const int32_t *qu, const int32_t *qv, int64_t j0,
                                  int64_t j1, uint8_t *ans, uint8_t *code, bool *overflowed, cudaStream_t s)
{
    uint32_t *cnt = c->d_counts;
    uint32_t *h = c->h_pinned;
    const SearchArgs a = search_args(ix, c, qu, qv, ans, code, cnt + kCntClaimed, cnt + kCntOverflow);
    cudaMemsetAsync(cnt + kCntSlots0, 0, sizeof(uint32_t) * 5, s);  // slots0, slots1, tasks, claimed, overflow
    // slot stamps are per wave (slots are cleared after each wave): level epochs 1, 2, ...
    uint32_t sep = 1;
    SlotList lists[2] = {{c->slot_list[0], cnt + kCntSlots0, c->table_slots},
                         {c->slot_list[1], cnt + kCntSlots1, c->table_slots}};
    qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
    k_search_setup<WD, WB><<<blocks_for(j1 - j0), kBlock, 0, s>>>(a, j0, j1, sep, lists[0]);
    ++ix->launches;
    qt_end(ix, c, s);
    int cur = 0;
    int64_t levels = 0;
    const int64_t max_levels = (int64_t)ix->n + 2;
    for (;;) {
        cudaMemcpyAsync(h, cnt, sizeof(uint32_t) * kCntWords, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return qfail(c, DBL_ERR_CUDA, std::string("search level: ") + cudaGetErrorString(e));
        if (h[kCntOverflow]) break;
        const uint32_t nslots = h[kCntSlots0 + cur];
        if (!nslots) break;
        if (++levels > max_levels) {
            ix->poisoned = true;
            return qfail(c, DBL_ERR_TIMEOUT, "search: level bound exceeded");
        }
        const int nxt = cur ^ 1;
        cudaMemsetAsync(cnt + kCntTasks, 0, sizeof(uint32_t), s);
        cudaMemsetAsync(cnt + kCntSlots0 + nxt, 0, sizeof(uint32_t), s);
        qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
        k_search_finalize<<<blocks_for(nslots), kBlock, 0, s>>>(a, lists[cur], cnt + kCntTasks);
        ++ix->launches;
        qt_begin(ix, c, DBL_KERNEL_SEARCH_EXPAND, s);
        ++sep;
        // tasks are at most nslots * (1 + maxdeg/kChunk); size the grid generously and let it stride
        launch_search_expand<WD, WB>(ix, c, a, (int64_t)nslots * 2, sep, lists[nxt], s);
        qt_end(ix, c, s);
        cur = nxt;
    }
    *overflowed = h[kCntOverflow] != 0;
    qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
    k_search_answer<<<blocks_for(j1 - j0), kBlock, 0, s>>>(a, j0, j1, *overflowed ? 0 : 1);
    ++ix->launches;
    k_search_clear<<<blocks_for(c->table_slots / 4), kBlock, 0, s>>>(a);
    ++ix->launches;
    qt_end(ix, c, s);
    atomic_add_host_stat(ix, 14, 1, s);
    atomic_add_host_stat(ix, 8, (uint64_t)levels, s);
    cudaError_t e = cudaGetLastError();
    return e ? qfail(c, DBL_ERR_CUDA, std::string("search wave: ") + cudaGetErrorString(e)) : DBL_OK;
}

template <int WD, int WB, int TEAM>
static dbl_status launch_search_persistent(dbl_index *ix, dbl_qctx *c, const int32_t *qu, const int32_t *qv,
                                           uint8_t *ans, uint8_t *code, cudaStream_t s)
{
    constexpr int kPB = pblock_of(hs_of(WD + WB));
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_search_persistent<WD, WB, TEAM>, kPB, 0);
    if (blocks_per_sm < 1) return qfail(c, DBL_ERR_CUDA, "persistent search: kernel does not fit on an SM");
    PersistState *ps = (PersistState *)c->pstate;
    cudaMemsetAsync(ps, 0, sizeof(PersistState), s);
    SearchArgs a = search_args(ix, c, qu, qv, ans, code, &ps->n_claimed, &ps->overflow);
    const uint32_t *n_und = c->d_counts + kCntUnd;
    GridBarrier bar = grid_barrier_at(c->d_counts);
    uint32_t *status = c->d_status;
    int64_t max_levels = (int64_t)ix->n + 2;
    void *args[] = {&a, &ps, &n_und, &bar, &status, &max_levels};
    dim3 grid((unsigned)num_sms()), block(kPB);
    qt_begin(ix, c, DBL_KERNEL_SEARCH_EXPAND, s);
    cudaError_t e =
        cudaLaunchCooperativeKernel((const void *)k_search_persistent<WD, WB, TEAM>, grid, block, args, 0, s);
    ++ix->launches;
    qt_end(ix, c, s);
    return e ? qfail(c, DBL_ERR_CUDA, std::string("persistent search launch: ") + cudaGetErrorString(e)) : DBL_OK;
}

template <int WD, int WB>
static dbl_status query_t(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                          uint8_t *code, cudaStream_t s)
{
    dbl_status st = ensure_search_scratch(c, q, s);
    if (st) return st;
    uint32_t *cnt = c->d_counts;
    cudaMemsetAsync(cnt + kCntUnd, 0, sizeof(uint32_t), s);
    // pairs per thread: option, else 4 for 32-byte records, 2 for 64, 1 for 128
    constexpr int HS = hs_of(WD + WB);
    int qpt = ix->opt.query_unroll ? ix->opt.query_unroll : (HS == 2 ? 4 : (HS == 4 ? 2 : 1));
    int64_t blocks = (q + (int64_t)kBlock * qpt - 1) / ((int64_t)kBlock * qpt);
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    qt_begin(ix, c, DBL_KERNEL_QUERY_LABEL, s);
    auto kern = qpt >= 4 ? k_query_label<WD, WB, 4> : (qpt == 2 ? k_query_label<WD, WB, 2> : k_query_label<WD, WB, 1>);
    kern<<<(unsigned)blocks, kBlock, 0, s>>>(u, v, q, ix->rec, ix->n, ans, code, c->und, cnt + kCntUnd, c->d_status,
                                             ix->d_stats);
    ++ix->launches;
    qt_end(ix, c, s);
    // one cooperative launch runs every wave, for the index's own context only
    // (cooperative grids of concurrent contexts would compete for residency)
    if ((ix->opt.flags & DBL_FLAG_PERSISTENT) && c == ix->qc) {
        switch (ix->opt.team) {
        case 4: st = launch_search_persistent<WD, WB, 4>(ix, c, u, v, ans, code, s); break;
        case 16:
        case 32: st = launch_search_persistent<WD, WB, 16>(ix, c, u, v, ans, code, s); break;
        default: st = launch_search_persistent<WD, WB, 8>(ix, c, u, v, ans, code, s); break;
        }
        return st;  // device errors (invalid ids, timeout) latch in the context's status word
    }
    uint32_t *h = c->h_pinned;
    cudaMemcpyAsync(h, cnt + kCntUnd, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h + 8, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return qfail(c, DBL_ERR_CUDA, std::string("query label test: ") + cudaGetErrorString(e));
    if (h[8]) {
        cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), s);  // consumed; nothing was changed
        return qfail(c, (dbl_status)h[8], "query: vertex id out of range");
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
        st = run_search_wave<WD, WB>(ix, c, u, v, r.j0, r.j1, ans, code, &over, s);
        if (st) return st;
        if (over) {
            const int64_t groups = (r.j1 - r.j0 + 63) / 64;
            if (groups <= 1) return qfail(c, DBL_ERR_CAPACITY, "search: one group overflowed the state table");
            const int64_t mid = r.j0 + (groups / 2) * 64;
            stack.push_back({mid, r.j1});
            stack.push_back({r.j0, mid});
        }
    }
    return DBL_OK;
}

dbl_status query(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                 uint8_t *code, cudaStream_t s)
{
    if (q == 0) return DBL_OK;
    const int key = ix->wd * 16 + ix->wb;
    switch (key) {
    case 1 * 16 + 1: return query_t<1, 1>(ix, c, u, v, q, ans, code, s);
    case 2 * 16 + 1: return query_t<2, 1>(ix, c, u, v, q, ans, code, s);
    case 1 * 16 + 2: return query_t<1, 2>(ix, c, u, v, q, ans, code, s);
    case 2 * 16 + 2: return query_t<2, 2>(ix, c, u, v, q, ans, code, s);
    case 4 * 16 + 1: return query_t<4, 1>(ix, c, u, v, q, ans, code, s);
    case 1 * 16 + 4: return query_t<1, 4>(ix, c, u, v, q, ans, code, s);
    case 2 * 16 + 4: return query_t<2, 4>(ix, c, u, v, q, ans, code, s);
    case 4 * 16 + 2: return query_t<4, 2>(ix, c, u, v, q, ans, code, s);
    case 4 * 16 + 4: return query_t<4, 4>(ix, c, u, v, q, ans, code, s);
    default: return qfail(c, DBL_ERR_INVALID, "unsupported (k, kprime) combination");
    }
}

size_t persist_state_bytes() { return sizeof(PersistState); }

}  // namespace dbl
