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
// pending for the next level.  All groups of a batch run in one wave, first
// in a slice of the table; if that overflows, the wave's found answers are
// kept and the rest rerun over the whole table, and if that overflows too,
// in halves.
#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_kernels.cuh"
#include "dbl_persistent.cuh"

namespace dbl {

// Words per half-record of a (WD, WB) instantiation; WD = WB = 0 marks the
// packed layout (k + k' <= 64: one word per half, DL in its low k bits, BL above).
__host__ __device__ constexpr int hs_of(int words) { return words == 0 ? 1 : (words <= 2 ? 2 : (words <= 4 ? 4 : 8)); }

// ------------------------------------------------------------ label test
// A pair is handled by LPP = HS / 2 adjacent lanes: lane `sub` of the group
// owns words 2*sub and 2*sub + 1 of each of the four half-records (DL_in |
// BL_in and DL_out | BL_out of u and of v) and loads them with one 16-byte
// load per half; the group's lanes together read each half as one contiguous
// request, and every lane holds the same registers whatever the label width
// (at 32-byte records the group is one lane).  Each lane evaluates Algorithm
// 2's label tests on its words, the partial verdicts are OR-ed across the
// group by shuffles, and lane 0 of the group writes the answer.  Each group
// takes QPT pairs (default 2) and issues all of their record loads before
// using any, so many DRAM sectors are in flight per warp; answers and codes
// are written coalesced, the deciding rules are counted per thread.  An
// undecided pair gets the answer byte kAnsUndecided; the search compacts those
// from the answer array itself (compact_undecided), so the label test writes
// nothing else (appending to an undecided list here, one atomic per warp,
// took a third of the kernel's time; one per block through a shared-memory
// stage still took a tenth).
constexpr uint8_t kAnsUndecided = 2;

template <int WD, int WB, int QPT>
__global__ void __launch_bounds__(kBlock) k_query_label(const int32_t *qu, const int32_t *qv, int64_t q,
                                                        const uint64_t *rec, int32_t n, uint8_t *ans,
                                                        uint8_t *code, uint32_t *status, unsigned long long *stats)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int LPP = HS / 2;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPP;
    const int w0 = 2 * sub;  // first word of this lane in every half
    unsigned int counts[6] = {0, 0, 0, 0, 0, 0};  // per group leader, by deciding rule (constant indices only)
    const int64_t groups = blockDim.x / LPP;      // pair slots per block and j
    const int64_t tile = groups * QPT;
    const int64_t stride = (int64_t)gridDim.x * tile;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < q; base += stride) {  // block-uniform
        int32_t u[QPT], v[QPT];
        bool live[QPT];
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const int64_t i = base + (int64_t)j * groups + threadIdx.x / LPP;
            live[j] = i < q;
            u[j] = live[j] ? __ldcs(qu + i) : 0;
            v[j] = live[j] ? __ldcs(qv + i) : 0;
        }
        ulonglong2 fu[QPT], bu[QPT], fv[QPT], bv[QPT];
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const bool ok = live[j] && (uint32_t)u[j] < (uint32_t)n && (uint32_t)v[j] < (uint32_t)n && u[j] != v[j];
            const int32_t uu = ok ? u[j] : 0, vv = ok ? v[j] : 0;
            if constexpr (HS == 2) {
                // a 32-byte record is one sector: one load for both halves
                load_rec32(rec + (size_t)uu * RW, fu[j].x, fu[j].y, bu[j].x, bu[j].y);
                load_rec32(rec + (size_t)vv * RW, fv[j].x, fv[j].y, bv[j].x, bv[j].y);
            } else {
                fu[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + (size_t)uu * RW + w0));
                bu[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + (size_t)uu * RW + HS + w0));
                fv[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + (size_t)vv * RW + w0));
                bv[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + (size_t)vv * RW + HS + w0));
            }
        }
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            // this lane's words: DL words are [0, WD), BL words [WD, WD + WB), the rest padding
            uint64_t uv = 0, vu = 0, su = 0, sv = 0, blf = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int w = w0 + h;
                const uint64_t a = h ? fu[j].y : fu[j].x, b = h ? bu[j].y : bu[j].x;
                const uint64_t c = h ? fv[j].y : fv[j].x, d = h ? bv[j].y : bv[j].x;
                if (w < WD) {
                    uv |= b & c;  // DL_out(u) & DL_in(v)
                    vu |= d & a;  // DL_out(v) & DL_in(u)
                    su |= b & a;
                    sv |= d & c;
                } else if (w < WD + WB) {
                    blf |= (a & ~c) | (d & ~b);  // BL_in(u) not in BL_in(v), BL_out(v) not in BL_out(u)
                }
            }
            uint32_t fl = (uv ? 1u : 0u) | (blf ? 2u : 0u) | (vu ? 4u : 0u) | ((su | sv) ? 8u : 0u);
#pragma unroll
            for (int o = 1; o < LPP; o <<= 1) fl |= __shfl_xor_sync(kFull, fl, o);
            const int64_t i = base + (int64_t)j * groups + threadIdx.x / LPP;
            uint8_t a = 0, c = DBL_CODE_UNDECIDED;
            if (live[j] && sub == 0) {
                if ((uint32_t)u[j] >= (uint32_t)n || (uint32_t)v[j] >= (uint32_t)n) {
                    set_status(status, DBL_ERR_INVALID);
                } else if (u[j] == v[j]) {
                    a = 1;
                    c = DBL_CODE_SELF;
                } else if (fl & 1u) {
                    a = 1;
                    c = DBL_CODE_DL;
                } else if (fl & 2u) {
                    c = DBL_CODE_BL;
                } else if (fl & 4u) {
                    c = DBL_CODE_THM1;
                } else if (fl & 8u) {
                    c = DBL_CODE_THM2;
                } else {
                    a = kAnsUndecided;
                }
                __stcs(ans + i, a);
                if (code) __stcs(code + i, c);
            }
#pragma unroll
            for (int r = 1; r < 6; ++r) counts[r] += (live[j] && sub == 0 && c == r) ? 1u : 0u;
        }
    }
#pragma unroll
    for (int r = 1; r < 6; ++r) {
        const unsigned int t = __reduce_add_sync(kFull, counts[r]);
        if (lane == 0 && t) atomicAdd(stats + r, (unsigned long long)t);
    }
}

// Label test of the packed layout (k + k' <= 64): a 16-byte record is the
// forward word and the backward word, DL in the bits of dlm and BL in the
// bits of blm; one lane per pair, QPT pairs per lane with all their loads in
// flight before any is used.  Same rules, order and outputs as k_query_label.
template <int QPT>
__global__ void __launch_bounds__(kBlock) k_query_label_packed(const int32_t *qu, const int32_t *qv, int64_t q,
                                                               const uint64_t *rec, int32_t n, uint64_t dlm,
                                                               uint64_t blm, uint8_t *ans, uint8_t *code,
                                                               uint32_t *status, unsigned long long *stats)
{
    const int lane = threadIdx.x & 31;
    unsigned int counts[6] = {0, 0, 0, 0, 0, 0};
    const int64_t tile = (int64_t)blockDim.x * QPT;
    const int64_t stride = (int64_t)gridDim.x * tile;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < q; base += stride) {
        int32_t u[QPT], v[QPT];
        bool live[QPT];
        ulonglong2 ru[QPT], rv[QPT];
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
            live[j] = i < q;
            u[j] = live[j] ? __ldcs(qu + i) : 0;
            v[j] = live[j] ? __ldcs(qv + i) : 0;
        }
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const bool ok = live[j] && (uint32_t)u[j] < (uint32_t)n && (uint32_t)v[j] < (uint32_t)n && u[j] != v[j];
            ru[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + 2 * (size_t)(ok ? u[j] : 0)));
            rv[j] = __ldcg(reinterpret_cast<const ulonglong2 *>(rec + 2 * (size_t)(ok ? v[j] : 0)));
        }
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const uint64_t a = ru[j].x, b = ru[j].y, c = rv[j].x, d = rv[j].y;  // fwd(u), bwd(u), fwd(v), bwd(v)
            const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
            uint8_t an = 0, cd = DBL_CODE_UNDECIDED;
            if (live[j]) {
                if ((uint32_t)u[j] >= (uint32_t)n || (uint32_t)v[j] >= (uint32_t)n) {
                    set_status(status, DBL_ERR_INVALID);
                } else if (u[j] == v[j]) {
                    an = 1;
                    cd = DBL_CODE_SELF;
                } else if (b & c & dlm) {                           // DL_out(u) & DL_in(v): Lemma 1
                    an = 1;
                    cd = DBL_CODE_DL;
                } else if (((a & ~c) | (d & ~b)) & blm) {           // BL containment fails: Lemma 2
                    cd = DBL_CODE_BL;
                } else if (d & a & dlm) {                           // DL_out(v) & DL_in(u): Theorem 1
                    cd = DBL_CODE_THM1;
                } else if (((b & a) | (d & c)) & dlm) {             // u or v with a landmark in its SCC: Theorem 2
                    cd = DBL_CODE_THM2;
                } else {
                    an = kAnsUndecided;
                }
                __stcs(ans + i, an);
                if (code) __stcs(code + i, cd);
            }
#pragma unroll
            for (int r = 1; r < 6; ++r) counts[r] += (live[j] && cd == r) ? 1u : 0u;
        }
    }
#pragma unroll
    for (int r = 1; r < 6; ++r) {
        const unsigned int t = __reduce_add_sync(kFull, counts[r]);
        if (lane == 0 && t) atomicAdd(stats + r, (unsigned long long)t);
    }
}

// The undecided pairs of a batch, from the answer array: und[] gets their
// indices (in no particular order) and *n_und their number.  The aligned
// middle of the array is read 16 bytes at a time, two words per thread and
// round (bytes compared four at a time), and each round's hits are written
// after one block-level reservation (the loop is block-uniform); the few
// bytes before the first and after the last aligned word are checked by
// block 0.
__device__ __forceinline__ uint32_t undecided_bits(uint32_t w)
{
    const uint32_t m = __vcmpeq4(w, 0x01010101u * kAnsUndecided);  // 0xff per matching byte
    return ((m >> 7) & 1u) | ((m >> 14) & 2u) | ((m >> 21) & 4u) | ((m >> 28) & 8u);
}

__device__ __forceinline__ void compact_undecided(const uint8_t *ans, int64_t q, int32_t *und, uint32_t *n_und)
{
    constexpr int K = 2;  // 16-byte words per thread and round
    int64_t head = (int64_t)((16u - ((uint32_t)(uintptr_t)ans & 15u)) & 15u);
    if (head > q) head = q;
    const int64_t nw = (q - head) / 16;
    const int64_t tail0 = head + nw * 16;
    const uint4 *wp = reinterpret_cast<const uint4 *>(ans + head);
    const int64_t tile = (int64_t)blockDim.x * K;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < nw; base += (int64_t)gridDim.x * tile) {
        uint32_t hits = 0;  // bit 16k + b: byte b of the thread's word k
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t wi = base + (int64_t)k * blockDim.x + threadIdx.x;
            if (wi < nw) {
                const uint4 w = __ldcg(wp + wi);
                hits |= (undecided_bits(w.x) | (undecided_bits(w.y) << 4) | (undecided_bits(w.z) << 8) |
                         (undecided_bits(w.w) << 12)) << (16 * k);
            }
        }
        uint32_t total = 0;
        uint32_t pos = block_reserve((uint32_t)__popc(hits), n_und, &total);
        while (hits) {
            const int bit = __ffs(hits) - 1;
            hits &= hits - 1;
            const int64_t wi = base + (int64_t)(bit >> 4) * blockDim.x + threadIdx.x;
            und[pos++] = (int32_t)(head + wi * 16 + (bit & 15));
        }
    }
    if (blockIdx.x == 0) {
        const int64_t extra = head + (q - tail0);  // fewer than 32
        if ((int64_t)threadIdx.x < extra) {
            const int64_t i = threadIdx.x < head ? (int64_t)threadIdx.x : tail0 + (threadIdx.x - head);
            if (ans[i] == kAnsUndecided) und[atomicAdd(n_und, 1u)] = (int32_t)i;
        }
    }
}

__global__ void k_compact_undecided(const uint8_t *ans, int64_t q, int32_t *und, uint32_t *n_und)
{
    compact_undecided(ans, q, und, n_und);
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
    uint64_t dlm, blm;  // packed labels: the DL and the BL bits of a half word
    uint64_t *qtab;
    unsigned long long *found;
    SearchCtx c;
    SearchTask *tasks;
    int64_t task_cap;
    int32_t *und;
    uint32_t *n_und;
    int64_t q;
    const int32_t *qu, *qv;
    uint8_t *ans, *code;
    unsigned long long *stats;
    int32_t *lists[2];
    int64_t list_cap;
    unsigned long long first_mask;  // slot mask of a wave's first attempt (kFirstSlots)
};

// Device-side state of the persistent search.
struct PersistState {
    uint32_t list_count[2];
    uint32_t task_count[2];
    uint32_t n_claimed;
    uint32_t overflow;
    int32_t top;
    int32_t pad;
    long long range[3];      // j0, j1, whole table (see kFirstSlots)
    long long stack[64][3];
};

// A wave first hashes its (group, vertex) states into the first kFirstSlots
// slots of the table (128 MB of slots: the pages stay in the address
// translation caches; dbl_options.search_first_log2 changes it); a wave that
// overflows them is rerun over the whole table, which always holds one group.
constexpr int64_t kFirstSlots = 1ll << 22;

constexpr int kMaxProbe = 2048;

// Claimed slots go to the block's claim stage (cst), flushed to c.claimed.
__device__ __forceinline__ IList claimed_list(const SearchCtx &c)
{
    return IList{c.claimed, c.n_claimed, (int64_t)c.slot_mask + 1, nullptr};  // each slot is claimed once per wave
}

__device__ __forceinline__ int64_t slot_find_or_insert(const SearchCtx &c, unsigned long long key, const IStage &cst)
{
    unsigned long long h = mix_key(key) & c.slot_mask;
    for (int p = 0; p < kMaxProbe; ++p) {
        SearchSlot *s = c.table + h;
        unsigned long long k = __ldcg(&s->key);
        if (k == key) return (int64_t)h;
        if (k == kEmptyKey) {
            unsigned long long prev = atomicCAS(&s->key, kEmptyKey, key);
            if (prev == kEmptyKey) {
                istage_push(cst, (int32_t)h, claimed_list(c));
                return (int64_t)h;
            }
            if (prev == key) return (int64_t)h;
        }
        h = (h + 1) & c.slot_mask;
    }
    atomicExch(c.overflow, 1u);
    return -1;
}

// qtab word layout per query: [u | v<<32][DL_out(u) x WD][BL_in(v) x WB][BL_out(v) x WB];
// packed labels: [u | v<<32][DL_out(u)][BL_in(v)][BL_out(v)], each a half word
// masked to its own bits (in place)
template <int WD, int WB>
struct QT {
    static constexpr int W = WD == 0 ? 4 : 1 + WD + 2 * WB;
};

__device__ __forceinline__ IList slot_list_of(const SearchCtx &c, const SlotList &l)
{
    return IList{l.items, l.count, l.cap, c.overflow};
}

// Slots that gain pending bits join the next level's list (through the block's
// list stage nst, flushed to `next`), once per level.
__device__ __forceinline__ void mark_pending(const SearchCtx &c, int64_t slot, unsigned long long bits,
                                             uint32_t epoch, const SlotList &next, const IStage &nst)
{
    SearchSlot *s = c.table + slot;
    atomicOr(&s->pend, bits);
    if (atomicExch(&s->stamp, epoch) != epoch) istage_push(nst, (int32_t)slot, slot_list_of(c, next));
}

// Wave setup: queries [j0, j1) of the undecided list (group j/64, bit j%64):
// fill the query table, zero the groups' found words, and emit the first
// level's tasks straight from each query's u: (u, g, chunk, bit j) for every
// chunk of Suc(u).  u itself is not entered in the visited table; if a search
// comes back to u it expands u once more, which adds nothing.  Each thread
// takes kSetupQ queries per round with all their loads in flight; the task
// list gets one reservation per block and round (the loop is block-uniform).
// Writes every lane's nch tasks (x, g, chunks 0 .. nch - 1, mask) from its
// position pos on, with the warp's lanes sharing the work (a lane whose
// vertex is a hub of thousands of chunks would otherwise write them alone,
// and the phase would wait for it); warp-collective.
__device__ __forceinline__ void warp_write_tasks(const SearchArgs &a, uint32_t nch, uint32_t pos, int32_t x,
                                                 uint32_t g, unsigned long long mask)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t excl = incl - nch;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t b0 = 0; b0 < total; b0 += 32) {  // warp-uniform
        const uint32_t e = b0 + lane;
        const int owner = flat_owner(excl, e);
        const uint32_t ch = e - __shfl_sync(kFull, excl, owner);
        const uint32_t p = __shfl_sync(kFull, pos, owner) + ch;
        const int32_t ox = __shfl_sync(kFull, x, owner);
        const uint32_t og = __shfl_sync(kFull, g, owner);
        const unsigned long long om = __shfl_sync(kFull, mask, owner);
        if (e >= total) continue;
        if ((int64_t)p >= a.task_cap) {
            atomicExch(a.c.overflow, 1u);
            continue;
        }
        SearchTask t;
        t.x = ox;
        t.g = og;
        t.chunk = ch;
        t.pad = 0;
        t.mask = om;
        a.tasks[p] = t;
    }
}

constexpr int kSetupQ = 4;

template <int WD, int WB>
__device__ __forceinline__ void search_setup(const SearchArgs &a, int64_t j0, int64_t j1, uint32_t *n_tasks)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gq = (j0 >> 6) + t0; gq < ((j1 + 63) >> 6); gq += nt) a.found[gq] = 0;
    const int64_t tile = (int64_t)blockDim.x * kSetupQ;
    for (int64_t base = j0 + (int64_t)blockIdx.x * tile; base < j1; base += (int64_t)gridDim.x * tile) {
        int64_t i[kSetupQ];
        int32_t u[kSetupQ], v[kSetupQ];
        uint32_t nch[kSetupQ], mine = 0;
#pragma unroll
        for (int k = 0; k < kSetupQ; ++k) {
            const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
            i[k] = j < j1 ? a.und[j] : -1;
        }
#pragma unroll
        for (int k = 0; k < kSetupQ; ++k) {
            u[k] = i[k] >= 0 ? a.qu[i[k]] : 0;
            v[k] = i[k] >= 0 ? a.qv[i[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < kSetupQ; ++k) {
            const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
            nch[k] = 0;
            if (i[k] < 0) continue;
            uint64_t *t = a.qtab + (size_t)j * W;
            t[0] = (uint64_t)(uint32_t)u[k] | ((uint64_t)(uint32_t)v[k] << 32);
            const uint64_t *ru = a.rec + (size_t)u[k] * RW, *rv = a.rec + (size_t)v[k] * RW;
            if constexpr (WD == 0) {  // packed: each label masked to its own bits
                t[1] = ru[1] & a.dlm;  // DL_out(u)
                t[2] = rv[0] & a.blm;  // BL_in(v)
                t[3] = rv[1] & a.blm;  // BL_out(v)
            } else {
#pragma unroll
                for (int w = 0; w < WD; ++w) t[1 + w] = ru[HS + w];  // DL_out(u)
#pragma unroll
                for (int w = 0; w < WB; ++w) {
                    t[1 + WD + w] = rv[WD + w];                       // BL_in(v)
                    t[1 + WD + WB + w] = rv[HS + WD + w];             // BL_out(v)
                }
            }
            nch[k] = (uint32_t)((deg_of(a.g, 0, u[k]) + kChunk - 1) / kChunk);
            mine += nch[k];
        }
        uint32_t total = 0;
        uint32_t pos = block_reserve(mine, n_tasks, &total);
        if (total == 0) continue;
#pragma unroll
        for (int k = 0; k < kSetupQ; ++k) {
            const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
            warp_write_tasks(a, nch[k], pos, u[k], (uint32_t)(j >> 6), 1ull << (j & 63));
            pos += nch[k];
        }
    }
}

// Slots listed for the next level -> tasks (x, g, chunk, mask) over Suc(x);
// one task-list reservation per block (the loop is block-uniform).
__device__ __forceinline__ void search_finalize(const SearchArgs &a, const SlotList &cur, uint32_t *n_tasks)
{
    const int64_t n = min((int64_t)ld_volatile_u32(cur.count), cur.cap);
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
        uint32_t total = 0;
        uint32_t pos = block_reserve(nch, n_tasks, &total);
        if (total == 0) continue;
        warp_write_tasks(a, nch, pos, x, (uint32_t)(key >> 32), mask);
    }
}

// One search level: for each task's edges x -> y and each live query j of the
// task's mask, in Algorithm 2's order: y == v_j -> found; DL prune; BL prune;
// otherwise y is visited for j, and bits new at y are pending for next level.
// Tests of one edge x -> y against the live queries m of group g (Algorithm
// 2's order) and the visit update of (g, y): returns the bits this thread
// set first in y's visit word (it owns their expansion from y), and the slot.
template <int WD, int WB>
__device__ __forceinline__ unsigned long long search_edge_visit(const SearchArgs &a, int32_t y, uint32_t g,
                                                                unsigned long long m, const IStage &cst,
                                                                int64_t &slot)
{
    constexpr int HS = hs_of(WD + WB);
    constexpr int RW = 2 * HS;
    constexpr int W = QT<WD, WB>::W;
    const uint64_t *qg = a.qtab + (size_t)g * 64 * W;
    uint64_t fy[HS], by[HS];
    if constexpr (HS == 2) {  // 32-byte records: one load for both halves
        load_rec32(a.rec + (size_t)y * RW, fy[0], fy[1], by[0], by[1]);
    } else {
        load_half<HS>(a.rec + (size_t)y * RW, fy);       // DL_in(y) | BL_in(y)
        load_half<HS>(a.rec + (size_t)y * RW + HS, by);  // DL_out(y) | BL_out(y)
    }
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
        if constexpr (WD == 0) {  // packed: the stored labels hold only their own bits
            dl = __ldg(qj + 1) & fy[0];
            if (dl) continue;
            bl = (fy[0] & a.blm & ~__ldg(qj + 2)) | (__ldg(qj + 3) & ~by[0]);
            if (bl) continue;
        } else {
#pragma unroll
            for (int w = 0; w < WD; ++w) dl |= __ldg(qj + 1 + w) & fy[w];
            if (dl) continue;
#pragma unroll
            for (int w = 0; w < WB; ++w)
                bl |= (fy[WD + w] & ~__ldg(qj + 1 + WD + w)) | (__ldg(qj + 1 + WD + WB + w) & ~by[WD + w]);
            if (bl) continue;
        }
        allowed |= bit;
    }
    if (hits) atomicOr(a.found + g, hits);
    slot = -1;
    if (!allowed) return 0;
    slot = slot_find_or_insert(a.c, ((unsigned long long)g << 32) | (uint32_t)y, cst);
    if (slot < 0) return 0;
    const unsigned long long old = atomicOr(&a.c.table[slot].visit, allowed);
    return allowed & ~old;
}

// search_edge_visit, with the new bits pending at (g, y) for the next level.
template <int WD, int WB>
__device__ __forceinline__ void search_edge(const SearchArgs &a, int32_t y, uint32_t g, unsigned long long m,
                                            uint32_t epoch, const SlotList &next, const IStage &cst,
                                            const IStage &nst)
{
    int64_t s;
    const unsigned long long nb = search_edge_visit<WD, WB>(a, y, g, m, cst, s);
    if (nb) mark_pending(a.c, s, nb, epoch, next, nst);
}

// Local continuation of the search (as in the label propagation): a state
// (g, y) whose new bits this warp owns and whose vertex has at most kChunk
// out-edges goes to the warp's list (shared memory) with y's adjacency range,
// and the warp expands its list in further rounds of the same level (up to
// kSLocalRounds), so chains of small vertices advance several hops per
// level; what is left after the last round becomes pending at its slot for
// the next level, as do states of larger vertices.  Each query bit of a
// state is still expanded exactly once: by the thread whose OR set it first.
struct SLocal {
    int32_t slot, y;
    uint32_t g;
    int32_t b0, o0;
    uint32_t deg;  // base degree | inserted degree << 16 (each at most kChunk)
    unsigned long long mask;
};
constexpr int kSLocal = 16;
constexpr int kSLocalRounds = 16;

// Warp-collective: lane-held new bits nb at slot s for (g, y) -> the warp's
// list or pending.
__device__ __forceinline__ void search_continue(const SearchArgs &a, unsigned long long nb, int64_t s, int32_t y,
                                                uint32_t g, uint32_t epoch, const SlotList &next, const IStage &nst,
                                                SLocal *wl, int &wl_n)
{
    const int lane = threadIdx.x & 31;
    AdjRange r{0, 0, 0, 0};
    if (nb) r = adj_of(a.g, 0, y);
    const int32_t d = r.bd + r.od;
    const bool loc = nb && d > 0 && d <= kChunk;
    const unsigned bl = __ballot_sync(kFull, loc);
    const int rank = __popc(bl & ((1u << lane) - 1u));
    const bool to_local = loc && wl_n + rank < kSLocal;
    if (to_local)
        wl[wl_n + rank] = SLocal{(int32_t)s, y, g, r.b0, r.o0, (uint32_t)r.bd | ((uint32_t)r.od << 16), nb};
    wl_n = min(kSLocal, wl_n + __popc(bl));
    if (nb && !to_local && d > 0) mark_pending(a.c, s, nb, epoch, next, nst);
}

// One flattened round: lane-held items (vertex x of group g, live bits m,
// x's adjacency r, edge range [lo, lo + cnt)); the warp walks the
// concatenation of the items' edges 32 at a time.
template <int WD, int WB>
__device__ __forceinline__ void search_round(const SearchArgs &a, uint32_t g, unsigned long long m, const AdjRange &r,
                                             uint32_t lo, uint32_t cnt, uint32_t epoch, const SlotList &next,
                                             const IStage &cst, const IStage &nst, SLocal *wl, int &wl_n,
                                             unsigned long long &relaxed)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t e = base + lane;
        const int owner = flat_owner(excl, e);
        const AdjRange orr{__shfl_sync(kFull, r.b0, owner), __shfl_sync(kFull, r.bd, owner),
                           __shfl_sync(kFull, r.o0, owner), 0};
        const uint32_t opos = __shfl_sync(kFull, lo, owner) + (e - __shfl_sync(kFull, excl, owner));
        const uint32_t og = __shfl_sync(kFull, g, owner);
        const unsigned long long om = __shfl_sync(kFull, m, owner);
        unsigned long long nb = 0;
        int64_t sl = -1;
        int32_t y = 0;
        if (e < total) {
            ++relaxed;
            y = adj_at(a.g, 0, orr, (int32_t)opos);
            nb = search_edge_visit<WD, WB>(a, y, og, om, cst, sl);
        }
        search_continue(a, nb, sl, y, og, epoch, next, nst, wl, wl_n);
    }
}

// Flattened search level (TEAM == 1): one task per lane per round, the warp
// walks the concatenation of its tasks' edges 32 at a time (see
// expand_level_flat), then the warp's local rounds.
template <int WD, int WB>
__device__ __forceinline__ void search_expand_flat(const SearchArgs &a, uint32_t n_tasks_in, uint32_t epoch,
                                                   const SlotList &next, const IStage &cst, const IStage &nst)
{
    __shared__ SLocal s_sl[32 * kSLocal];
    const int lane = threadIdx.x & 31;
    SLocal *wl = s_sl + (threadIdx.x >> 5) * kSLocal;
    int wl_n = 0;  // warp-uniform
    const int64_t ntasks = min((int64_t)n_tasks_in, a.task_cap);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long relaxed = 0;
    for (int64_t r0 = 0; warp + nwarps * r0 < ntasks; r0 += 32) {  // warp-uniform
        const int64_t t = warp + nwarps * (r0 + lane);
        AdjRange r{0, 0, 0, 0};
        uint32_t lo = 0, cnt = 0, g = 0;
        unsigned long long m = 0;
        if (t < ntasks) {
            const SearchTask tk = a.tasks[t];
            m = tk.mask & ~__ldcg(a.found + tk.g);
            if (m) {
                r = adj_of(a.g, 0, tk.x);
                g = tk.g;
                const int32_t d = r.bd + r.od;
                lo = tk.chunk * (uint32_t)kChunk;
                const int32_t hi = min(d, (int32_t)lo + kChunk);
                cnt = hi > (int32_t)lo ? (uint32_t)(hi - (int32_t)lo) : 0u;
            }
        }
        search_round<WD, WB>(a, g, m, r, lo, cnt, epoch, next, cst, nst, wl, wl_n, relaxed);
    }
    for (int lr = 0; lr < kSLocalRounds && wl_n > 0; ++lr) {
        __syncwarp();
        const bool has = lane < wl_n;
        const SLocal it = has ? wl[lane] : SLocal{0, 0, 0u, 0, 0, 0u, 0ull};
        __syncwarp();
        wl_n = 0;
        unsigned long long m = 0;
        AdjRange r{0, 0, 0, 0};
        uint32_t cnt = 0;
        if (has) {
            m = it.mask & ~__ldcg(a.found + it.g);
            if (m) {
                r = AdjRange{it.b0, (int32_t)(it.deg & 0xffffu), it.o0, (int32_t)(it.deg >> 16)};
                cnt = (uint32_t)(r.bd + r.od);
            }
        }
        search_round<WD, WB>(a, it.g, m, r, 0u, cnt, epoch, next, cst, nst, wl, wl_n, relaxed);
    }
    __syncwarp();
    if (lane < wl_n) {  // left for the next level
        const SLocal it = wl[lane];
        mark_pending(a.c, it.slot, it.mask, epoch, next, nst);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) relaxed += __shfl_xor_sync(kFull, relaxed, o);
    if (lane == 0 && relaxed) atomicAdd(a.stats + 10, relaxed);
    istage_flush(cst, claimed_list(a.c));
    istage_flush(nst, slot_list_of(a.c, next));
}

template <int WD, int WB, int TEAM>
__device__ __forceinline__ void search_expand(const SearchArgs &a, uint32_t n_tasks_in, uint32_t epoch,
                                              const SlotList &next, const IStage &cst, const IStage &nst)
{
    if constexpr (TEAM == 1) {
        search_expand_flat<WD, WB>(a, n_tasks_in, epoch, next, cst, nst);
    } else {
        // TEAM lanes per task, 32/TEAM tasks per warp at a time
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
            for (int32_t e = lo + tl; e < hi; e += TEAM) {
                ++relaxed;
                search_edge<WD, WB>(a, adj_at(a.g, 0, r, e), tk.g, m, epoch, next, cst, nst);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) relaxed += __shfl_xor_sync(kFull, relaxed, o);
        if (lane == 0 && relaxed) atomicAdd(a.stats + 10, relaxed);
        istage_flush(cst, claimed_list(a.c));
        istage_flush(nst, slot_list_of(a.c, next));
    }
}

// Answers of queries [j0, j1): found -> true (bfs_pos); otherwise false
// (bfs_neg) when the wave ran to exhaustion (final), else left for a rerun.
// Four queries per thread and round, loads first.
__device__ __forceinline__ void search_answer(const SearchArgs &a, int64_t j0, int64_t j1, bool final_wave)
{
    constexpr int Q = 4;
    __shared__ unsigned int cnt[2];
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockDim.x * Q;
    for (int64_t base = j0 + (int64_t)blockIdx.x * tile; base < j1; base += (int64_t)gridDim.x * tile) {
        int64_t i[Q];
        bool hit[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
            i[k] = j < j1 ? a.und[j] : -1;
            hit[k] = j < j1 && ((__ldcg(a.found + (j >> 6)) >> (j & 63)) & 1ull);
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if (i[k] < 0) continue;
            if (hit[k]) {
                a.ans[i[k]] = 1;
                if (a.code) a.code[i[k]] = DBL_CODE_BFS_POS;
                atomicAdd(&cnt[0], 1u);
            } else if (final_wave) {
                a.ans[i[k]] = 0;
                if (a.code) a.code[i[k]] = DBL_CODE_BFS_NEG;
                atomicAdd(&cnt[1], 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt[0]) atomicAdd(a.stats + DBL_CODE_BFS_POS, (unsigned long long)cnt[0]);
        if (cnt[1]) atomicAdd(a.stats + DBL_CODE_BFS_NEG, (unsigned long long)cnt[1]);
    }
}

// Return every slot claimed in the wave to empty (four per thread and round).
__device__ __forceinline__ void search_clear(const SearchArgs &a)
{
    constexpr int Q = 4;
    const int64_t n = ld_volatile_u32(a.c.n_claimed);
    const int64_t tile = (int64_t)blockDim.x * Q;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        int32_t sl[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
            sl[k] = i < n ? a.c.claimed[i] : -1;
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if (sl[k] < 0) continue;
            SearchSlot *s = a.c.table + sl[k];
            s->key = kEmptyKey;
            s->visit = 0;
            s->pend = 0;
            s->stamp = 0;
        }
    }
}

// ------------------------------------------------------------ per-level kernels
template <int WD, int WB>
__global__ void k_search_setup(SearchArgs a, int64_t j0, int64_t j1, uint32_t *n_tasks)
{
    search_setup<WD, WB>(a, j0, j1, n_tasks);
}

__global__ void k_search_finalize(SearchArgs a, SlotList cur, uint32_t *n_tasks) { search_finalize(a, cur, n_tasks); }

template <int WD, int WB, int TEAM>
__global__ void __launch_bounds__(kBlock) k_search_expand(SearchArgs a, const uint32_t *n_tasks, uint32_t epoch,
                                                          SlotList next)
{
    DBL_BLOCK_ISTAGE(cst);
    DBL_BLOCK_ISTAGE(nst);
    search_expand<WD, WB, TEAM>(a, ld_volatile_u32(n_tasks), epoch, next, cst, nst);
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
// Per level: finalize, barrier, expand, barrier.  An overflowing wave over
// the first slots is rerun over the whole table, one over the whole table in
// halves.
template <int WD, int WB, int TEAM>
__device__ __forceinline__ void search_waves(const SearchArgs &a, PersistState *ps, const uint32_t *n_und,
                                             GridSync &gs, uint32_t *status, int64_t max_levels, const IStage &cst,
                                             const IStage &nst)
{
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    compact_undecided(a.ans, a.q, a.und, a.n_und);
    if (!gs.sync(status)) return;
    const uint32_t U = ld_volatile_u32(n_und);
    if (U == 0) return;
    if (leader) {
        ps->top = 1;
        ps->stack[0][0] = 0;
        ps->stack[0][1] = U;
        ps->stack[0][2] = 0;
    }
    unsigned long long levels = 0, waves = 0;
    for (;;) {
        if (leader) {
            if (ps->top > 0) {
                --ps->top;
                ps->range[0] = ps->stack[ps->top][0];
                ps->range[1] = ps->stack[ps->top][1];
                ps->range[2] = ps->stack[ps->top][2];
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
        const bool whole = *(volatile long long *)&ps->range[2] != 0;
        SearchArgs aw = a;
        if (!whole) aw.c.slot_mask = a.first_mask;
        ++waves;
        SlotList lists[2] = {{a.lists[0], &ps->list_count[0], a.list_cap}, {a.lists[1], &ps->list_count[1], a.list_cap}};
        search_setup<WD, WB>(aw, j0, j1, &ps->task_count[0]);
        if (!gs.sync(status)) return;
        // level L: expand task list L%2 into slot list L%2 (slot stamps L+2),
        // then turn that slot list into task list (L+1)%2
        for (int64_t L = 0;; ++L) {
            const int cur = (int)(L & 1);
            const uint32_t ntk = ld_volatile_u32(&ps->task_count[cur]);
            if (!ntk || ld_volatile_u32(&ps->overflow) || ld_volatile_u32(status)) break;
            if (L >= max_levels) {
                set_status(status, DBL_ERR_TIMEOUT);
                break;
            }
            ++levels;
            if (leader) ps->task_count[cur ^ 1] = 0;
            search_expand<WD, WB, TEAM>(aw, ntk, (uint32_t)(L + 2), lists[cur], cst, nst);
            if (!gs.sync(status)) return;
            if (!ld_volatile_u32(&ps->list_count[cur]) || ld_volatile_u32(&ps->overflow)) break;
            search_finalize(aw, lists[cur], &ps->task_count[cur ^ 1]);
            if (!gs.sync(status)) return;
            if (leader) ps->list_count[cur] = 0;  // written again two levels on, after a barrier
        }
        const bool over = ld_volatile_u32(&ps->overflow) != 0;
        search_answer(aw, j0, j1, !over);
        search_clear(aw);
        if (!gs.sync(status)) return;
        if (over && leader) {
            const long long groups = (j1 - j0 + 63) / 64;
            if (!whole && a.first_mask < a.c.slot_mask && ps->top < 64) {
                ps->stack[ps->top][0] = j0;  // rerun over the whole table
                ps->stack[ps->top][1] = j1;
                ps->stack[ps->top][2] = 1;
                ps->top += 1;
            } else if (groups <= 1 || ps->top + 2 > 64) {
                set_status(status, DBL_ERR_CAPACITY);
            } else {
                const long long mid = j0 + (groups / 2) * 64;
                ps->stack[ps->top][0] = mid;
                ps->stack[ps->top][1] = j1;
                ps->stack[ps->top][2] = whole ? 1 : 0;
                ps->stack[ps->top + 1][0] = j0;
                ps->stack[ps->top + 1][1] = mid;
                ps->stack[ps->top + 1][2] = whole ? 1 : 0;
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
    DBL_BLOCK_ISTAGE(cst);
    DBL_BLOCK_ISTAGE(nst);
    search_waves<WD, WB, TEAM>(a, ps, n_und, gs, status, max_levels, cst, nst);
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

static SearchArgs search_args(dbl_index *ix, dbl_qctx *c, const int32_t *qu, const int32_t *qv, int64_t q,
                              uint8_t *ans, uint8_t *code, uint32_t *n_claimed, uint32_t *overflow)
{
    SearchArgs a;
    a.g = dev_graph(ix);
    a.rec = ix->rec;
    a.dlm = ix->dl_mask;
    a.blm = ix->bl_mask;
    a.qtab = c->qtab;
    a.found = c->found;
    a.c = SearchCtx{c->table, (unsigned long long)(c->table_slots - 1), c->claimed, n_claimed, overflow};
    a.tasks = c->stask;
    a.task_cap = c->stask_cap;
    a.und = c->und;
    a.n_und = c->d_counts + kCntUnd;
    a.q = q;
    a.qu = qu;
    a.qv = qv;
    a.ans = ans;
    a.code = code;
    a.stats = ix->d_stats;
    a.lists[0] = c->slot_list[0];
    a.lists[1] = c->slot_list[1];
    a.list_cap = c->table_slots;
    const int64_t first = ix->opt.search_first_log2 > 0 ? (1ll << std::min(ix->opt.search_first_log2, 40)) : kFirstSlots;
    a.first_mask = (unsigned long long)(std::min<int64_t>(c->table_slots, first) - 1);
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
    case 1: k_search_expand<WD, WB, 1><<<blocks_for(est * 4), kBlock, 0, s>>>(a, nt, sep, next); break;
    case 4: k_search_expand<WD, WB, 4><<<blocks_for(est * 4), kBlock, 0, s>>>(a, nt, sep, next); break;
    case 16:
    case 32: k_search_expand<WD, WB, 16><<<blocks_for(est * 16), kBlock, 0, s>>>(a, nt, sep, next); break;
    default: k_search_expand<WD, WB, 8><<<blocks_for(est * 8), kBlock, 0, s>>>(a, nt, sep, next); break;
    }
    ++ix->launches;
}

template <int WD, int WB>
static dbl_status run_search_wave(dbl_index *ix, dbl_qctx *c, const int32_t *qu, const int32_t *qv, int64_t j0,
                                  int64_t j1, bool whole, uint8_t *ans, uint8_t *code, bool *overflowed,
                                  cudaStream_t s)
{
    uint32_t *cnt = c->d_counts;
    uint32_t *h = c->h_pinned;
    SearchArgs a = search_args(ix, c, qu, qv, 0, ans, code, cnt + kCntClaimed, cnt + kCntOverflow);
    if (!whole) a.c.slot_mask = a.first_mask;
    cudaMemsetAsync(cnt + kCntSlots0, 0, sizeof(uint32_t) * 5, s);  // slots0, slots1, tasks, claimed, overflow
    SlotList lists[2] = {{c->slot_list[0], cnt + kCntSlots0, c->table_slots},
                         {c->slot_list[1], cnt + kCntSlots1, c->table_slots}};
    qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
    k_search_setup<WD, WB><<<blocks_for((j1 - j0 + kSetupQ - 1) / kSetupQ), kBlock, 0, s>>>(a, j0, j1, cnt + kCntTasks);
    ++ix->launches;
    qt_end(ix, c, s);
    // level L: expand the task list into slot list L%2 (slot stamps L+2; slots
    // are cleared after each wave), then turn that slot list into the next
    // task list.  One host round trip per level reads the task count.
    int64_t levels = 0;
    const int64_t max_levels = (int64_t)ix->n + 2;
    for (int64_t L = 0;; ++L) {
        cudaMemcpyAsync(h, cnt, sizeof(uint32_t) * kCntWords, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return qfail(c, DBL_ERR_CUDA, std::string("search level: ") + cudaGetErrorString(e));
        if (h[kCntOverflow]) break;
        const uint32_t ntasks = h[kCntTasks];
        if (!ntasks) break;
        if (++levels > max_levels) {
            ix->poisoned = true;
            return qfail(c, DBL_ERR_TIMEOUT, "search: level bound exceeded");
        }
        const int cur = (int)(L & 1);
        cudaMemsetAsync(cnt + kCntSlots0 + cur, 0, sizeof(uint32_t), s);
        qt_begin(ix, c, DBL_KERNEL_SEARCH_EXPAND, s);
        launch_search_expand<WD, WB>(ix, c, a, (int64_t)ntasks, (uint32_t)(L + 2), lists[cur], s);
        qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
        cudaMemsetAsync(cnt + kCntTasks, 0, sizeof(uint32_t), s);
        // the slot count is on the device: a fixed grid strides over it
        k_search_finalize<<<(unsigned)(num_sms() * 8), kBlock, 0, s>>>(a, lists[cur], cnt + kCntTasks);
        ++ix->launches;
        qt_end(ix, c, s);
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
                                           int64_t q, uint8_t *ans, uint8_t *code, cudaStream_t s)
{
    constexpr int kPB = pblock_of(hs_of(WD + WB));
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_search_persistent<WD, WB, TEAM>, kPB, 0);
    if (blocks_per_sm < 1) return qfail(c, DBL_ERR_CUDA, "persistent search: kernel does not fit on an SM");
    // every field is written by block 0 before any block reads it (after the
    // first grid barrier), so the state needs no clearing here
    PersistState *ps = (PersistState *)c->pstate;
    SearchArgs a = search_args(ix, c, qu, qv, q, ans, code, &ps->n_claimed, &ps->overflow);
    const uint32_t *n_und = c->d_counts + kCntUnd;
    GridBarrier bar = grid_barrier_at(c->d_counts);
    if ((ix->opt.flags & DBL_FLAG_TIMING) && c == ix->qc) bar.trace = ix->d_trace;
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
    // pairs per lane group: option, else 2 at 32-byte records (2 beats 4:
    // more resident warps, and 1: fewer loads in flight) and 4 at wider ones
    // (64-byte records: 4 -> 374 us, 2 -> 407 us, 1 -> 477 us per 10M pairs;
    // 128-byte: 4 and 1 -> 523 us, 2 -> 559 us); a group of HS / 2 lanes
    // keeps the same registers at every record width
    constexpr int HS = hs_of(WD + WB);
    const int qpt = ix->opt.query_unroll ? ix->opt.query_unroll : (HS == 2 ? 2 : 4);
    const int64_t pairs_per_block = (int64_t)(kBlock / (HS >= 2 ? HS / 2 : 1)) * qpt;
    int64_t blocks = (q + pairs_per_block - 1) / pairs_per_block;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    qt_begin(ix, c, DBL_KERNEL_QUERY_LABEL, s);
    if constexpr (WD == 0) {
        auto kern = qpt >= 4 ? k_query_label_packed<4> : (qpt == 2 ? k_query_label_packed<2> : k_query_label_packed<1>);
        kern<<<(unsigned)blocks, kBlock, 0, s>>>(u, v, q, ix->rec, ix->n, ix->dl_mask, ix->bl_mask, ans, code,
                                                 c->d_status, ix->d_stats);
    } else {
        auto kern =
            qpt >= 4 ? k_query_label<WD, WB, 4> : (qpt == 2 ? k_query_label<WD, WB, 2> : k_query_label<WD, WB, 1>);
        kern<<<(unsigned)blocks, kBlock, 0, s>>>(u, v, q, ix->rec, ix->n, ans, code, c->d_status, ix->d_stats);
    }
    ++ix->launches;
    qt_end(ix, c, s);
    // one cooperative launch runs every wave, for the index's own context only
    // (cooperative grids of concurrent contexts would compete for residency)
    if ((ix->opt.flags & DBL_FLAG_PERSISTENT) && c == ix->qc) {
        switch (ix->opt.team) {
        case 1: st = launch_search_persistent<WD, WB, 1>(ix, c, u, v, q, ans, code, s); break;
        case 4: st = launch_search_persistent<WD, WB, 4>(ix, c, u, v, q, ans, code, s); break;
        case 16:
        case 32: st = launch_search_persistent<WD, WB, 16>(ix, c, u, v, q, ans, code, s); break;
        default: st = launch_search_persistent<WD, WB, 8>(ix, c, u, v, q, ans, code, s); break;
        }
        return st;  // device errors (invalid ids, timeout) latch in the context's status word
    }
    qt_begin(ix, c, DBL_KERNEL_SEARCH_OTHER, s);
    k_compact_undecided<<<blocks_for((q + 31) / 32), kBlock, 0, s>>>(ans, q, c->und, cnt + kCntUnd);
    ++ix->launches;
    qt_end(ix, c, s);
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
    // waves: all groups at once in the first slots; on overflow the
    // unanswered rerun over the whole table, then in halves
    const int64_t first_slots = std::min<int64_t>(
        c->table_slots, ix->opt.search_first_log2 > 0 ? (1ll << std::min(ix->opt.search_first_log2, 40)) : kFirstSlots);
    struct Range {
        int64_t j0, j1;
        bool whole;
    };
    std::vector<Range> stack{{0, U, false}};
    while (!stack.empty()) {
        Range r = stack.back();
        stack.pop_back();
        bool over = false;
        st = run_search_wave<WD, WB>(ix, c, u, v, r.j0, r.j1, r.whole, ans, code, &over, s);
        if (st) return st;
        if (over) {
            const int64_t groups = (r.j1 - r.j0 + 63) / 64;
            if (!r.whole && first_slots < c->table_slots) {
                stack.push_back({r.j0, r.j1, true});
                continue;
            }
            if (groups <= 1) return qfail(c, DBL_ERR_CAPACITY, "search: one group overflowed the state table");
            const int64_t mid = r.j0 + (groups / 2) * 64;
            stack.push_back({mid, r.j1, r.whole});
            stack.push_back({r.j0, mid, r.whole});
        }
    }
    return DBL_OK;
}

dbl_status query(dbl_index *ix, dbl_qctx *c, const int32_t *u, const int32_t *v, int64_t q, uint8_t *ans,
                 uint8_t *code, cudaStream_t s)
{
    if (q == 0) return DBL_OK;
    if (ix->packed) return query_t<0, 0>(ix, c, u, v, q, ans, code, s);
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
