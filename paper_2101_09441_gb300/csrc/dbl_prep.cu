// Graph preparation, landmark / leaf selection and label seeding.
//
//   prep_graph       copy CSR-out, validate it, build CSR-in (the reverse
//                    graph G' of Section 2) by count / scan / scatter.
//   select_landmarks top-k by M(u) = |Pre(u)| * |Suc(u)| (Section 4.1), ties
//                    by smaller id: an 8-bit radix select finds the k-th
//                    value T on the device, then the vertices above T and the
//                    first ties in id order are ranked in one block.
//   select_leaves    zero in-degree -> seeds BL_in, zero out-degree -> seeds
//                    BL_out (Definition 2); bucket by Fibonacci hashing.
//   seed_labels      a landmark / leaf labels itself (Figure 1 shows
//                    v5 in DL_in(v5) and v1 in BL_in(v1)); every vertex with
//                    a non-zero half starts the frontier.
#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_kernels.cuh"

namespace dbl {

// ------------------------------------------------------------ scan
constexpr int kScanItems = 4;
constexpr int kScanTile = kBlock * kScanItems;

// Exclusive block scan of one value per thread; *total (shared) gets the sum.
__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t *total)
{
    constexpr int NW = kBlock / 32;
    __shared__ int64_t warp_sums[NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t sv = lane < NW ? warp_sums[lane] : 0;
        int64_t si = sv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(kFull, si, o);
            if (lane >= o) si += t;
        }
        if (lane < NW) warp_sums[lane] = si - sv;
        if (lane == NW - 1) *total = si;
    }
    __syncthreads();
    int64_t r = warp_sums[wid] + incl - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_tile_sums(const int32_t *in, int64_t n, int64_t *tile_sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
        if (j < n) s += in[j];
    }
    __shared__ int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tile_offsets(int64_t *tile_sums, int64_t ntiles)
{
    // one block: exclusive scan in place, in chunks of kBlock
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += kBlock) {
        int64_t j = base + threadIdx.x;
        int64_t x = j < ntiles ? tile_sums[j] : 0;
        int64_t e = block_excl_scan(x, &tot);
        if (j < ntiles) tile_sums[j] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int32_t *in, int32_t *out, int64_t n, const int64_t *tile_offs)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + i;
        v[i] = j < n ? in[j] : 0;
        s += v[i];
    }
    __shared__ int64_t tot;
    int64_t e = block_excl_scan(s, &tot) + tile_offs[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + i;
        if (j < n) out[j] = (int32_t)e;
        e += v[i];
    }
}

dbl_status exclusive_scan_i32(dbl_index *ix, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return DBL_OK;
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t *tiles = nullptr;
    dbl_status st = alloc_buf(ix, (void **)&tiles, sizeof(int64_t) * (size_t)ntiles, s);
    if (st) return st;
    k_scan_tile_sums<<<(unsigned)ntiles, kBlock, 0, s>>>(in, n, tiles);
    ++ix->launches;
    k_scan_tile_offsets<<<1, kBlock, 0, s>>>(tiles, ntiles);
    ++ix->launches;
    k_scan_apply<<<(unsigned)ntiles, kBlock, 0, s>>>(in, out, n, tiles);
    ++ix->launches;
    free_buf(ix, tiles, s);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(ix, e, "scan") : DBL_OK;
}

// ------------------------------------------------------------ graph prep
__global__ void k_validate_csr(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t m,
                               uint32_t *status)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= (int64_t)n; i += stride) {
        int32_t r = row_ptr[i];
        if (i == 0 && r != 0) set_status(status, DBL_ERR_INVALID);
        if (i == n && (int64_t)r != m) set_status(status, DBL_ERR_INVALID);
        if (i < n && row_ptr[i + 1] < r) set_status(status, DBL_ERR_INVALID);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        int32_t c = col[e];
        if (c < 0 || c >= n) set_status(status, DBL_ERR_INVALID);
    }
}

__global__ void k_count_in(const int32_t *col, int64_t m, int32_t *indeg)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(indeg + col[e], 1);
}

// ------------------------------------------------------------ balanced row walks
// Rows below kHeavyDeg edges are walked by warps, 32 rows at a time, and the
// longer ones by a block each, so that no warp is left with a hub's row (the
// largest R-MAT rows hold hundreds of thousands of edges).
constexpr int32_t kHeavyDeg = 1024;

constexpr int kWalkUnroll = 4;  // edges per lane in flight in the row walks

// Exclusive prefix of the lanes' row lengths and their total.
__device__ __forceinline__ uint32_t walk_prefix(int32_t deg, uint32_t &total)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = (uint32_t)deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(kFull, incl, 31);
    return incl - (uint32_t)deg;
}

// The warp walks the concatenation of its lanes' rows (lane l: a row of
// length deg_l from position start_l; excl its exclusive prefix), U x 32 edges
// per step: edge e = base + 32k + lane (k < U) is at position p[k] of lane
// owner[k]'s row, ok[k] when e is below the total.  Every lane of the warp
// calls it.
template <int U>
__device__ __forceinline__ void walk_step(uint32_t excl, int32_t start, uint32_t base, uint32_t total, int owner[U],
                                          int32_t p[U], bool ok[U])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint32_t e = base + 32u * k + lane;
        owner[k] = flat_owner(excl, e);
        const int32_t ostart = __shfl_sync(kFull, start, owner[k]);
        const uint32_t oexcl = __shfl_sync(kFull, excl, owner[k]);
        ok[k] = e < total;
        p[k] = ostart + (int32_t)(e - oexcl);
    }
}

// scatter u into Pre(col[p]) for every edge u -> col[p]; rows of kHeavyDeg
// edges or more go to the heavy list (k_scatter_in_heavy).  The column loads,
// then the cursor increments, then the stores of a step are issued together.
__global__ void k_scatter_in(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t *cursor,
                             int32_t *in_col, int32_t *heavy, uint32_t *nheavy)
{
    constexpr int U = kWalkUnroll;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = w * 32; r0 < n; r0 += nw * 32) {  // warp-uniform
        const int64_t u = r0 + lane;
        int32_t b = 0, d = 0;
        if (u < n) {
            b = row_ptr[u];
            d = row_ptr[u + 1] - b;
        }
        if (d >= kHeavyDeg) {
            heavy[atomicAdd(nheavy, 1u)] = (int32_t)u;
            d = 0;
        }
        uint32_t total;
        const uint32_t excl = walk_prefix(d, total);
        for (uint32_t base = 0; base < total; base += 32u * U) {
            int owner[U];
            int32_t p[U], v[U], pos[U];
            bool ok[U];
            walk_step<U>(excl, b, base, total, owner, p, ok);
#pragma unroll
            for (int k = 0; k < U; ++k) v[k] = ok[k] ? col[p[k]] : 0;
#pragma unroll
            for (int k = 0; k < U; ++k) pos[k] = ok[k] ? atomicAdd(cursor + v[k], 1) : 0;
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (ok[k]) in_col[pos[k]] = (int32_t)(r0 + owner[k]);
        }
    }
}

__global__ void k_scatter_in_heavy(const int32_t *row_ptr, const int32_t *col, int32_t *cursor, int32_t *in_col,
                                   const int32_t *heavy, const uint32_t *nheavy)
{
    constexpr int U = kWalkUnroll;
    const uint32_t nh = *nheavy;
    for (uint32_t i = blockIdx.x; i < nh; i += gridDim.x) {
        const int32_t u = heavy[i];
        const int32_t e = row_ptr[u + 1];
        for (int32_t p0 = row_ptr[u] + (int32_t)threadIdx.x; p0 < e; p0 += U * (int32_t)blockDim.x) {
            int32_t v[U], pos[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int32_t p = p0 + k * (int32_t)blockDim.x;
                v[k] = p < e ? col[p] : -1;
            }
#pragma unroll
            for (int k = 0; k < U; ++k) pos[k] = v[k] >= 0 ? atomicAdd(cursor + v[k], 1) : 0;
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (v[k] >= 0) in_col[pos[k]] = u;
        }
    }
}

// Per-vertex adjacency metadata from the two CSRs (no inserted edges yet):
// vertex x's inserted edges start in its slots0 reserved pool entries at
// x * slots0 (both pools), empty.
__global__ void k_fill_vmeta(const int32_t *out_ptr, const int32_t *in_ptr, int32_t n, int32_t slots0, VMeta *vm,
                             uint32_t *status)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o0 = out_ptr[x], od = out_ptr[x + 1] - o0;
        const int32_t i0 = in_ptr[x], id = in_ptr[x + 1] - i0;
        if (od >= (1 << kDegBits) || id >= (1 << kDegBits)) set_status(status, DBL_ERR_INVALID);
        const int32_t off = (int32_t)(x * slots0);
        VMeta v;
        v.d[0] = VAdj{o0, va_dc(od, slots0), off, 0};
        v.d[1] = VAdj{i0, va_dc(id, slots0), off, 0};
        vm[x] = v;
    }
}

// Rows [v0, v0 + c) of vertices added later: no edges, their reserved slots.
__global__ void k_init_vmeta_rows(int32_t v0, int32_t c, int32_t slots0, VMeta *vm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = v0 + i;
        const int32_t off = (int32_t)(x * slots0);
        VMeta v;
        v.d[0] = VAdj{0, va_dc(0, slots0), off, 0};
        v.d[1] = VAdj{0, va_dc(0, slots0), off, 0};
        vm[x] = v;
    }
}

static unsigned grid_for(int64_t work, int per_block = kBlock)
{
    int64_t b = (work + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void init_vmeta_rows(dbl_index *ix, int32_t v0, int32_t c, cudaStream_t s)
{
    k_init_vmeta_rows<<<grid_for(c), kBlock, 0, s>>>(v0, c, ix->slots0, ix->vm);
    ++ix->launches;
}

dbl_status prep_graph(dbl_index *ix, const dbl_graph *g, cudaStream_t s)
{
    const int32_t n = ix->n;
    const int64_t m = ix->m;
    cudaError_t e;
    e = cudaMemcpyAsync(ix->out_ptr, g->row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s);
    if (e) return cuda_fail(ix, e, "copy row_ptr");
    if (m) {
        e = cudaMemcpyAsync(ix->out_col, g->col, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, s);
        if (e) return cuda_fail(ix, e, "copy col");
    }
    k_validate_csr<<<grid_for(m > n ? m : n + 1), kBlock, 0, s>>>(ix->out_ptr, ix->out_col, n, m, ix->d_status);
    ++ix->launches;
    dbl_status st = read_status(ix, s);
    if (st) return fail(ix, st, "invalid CSR: row_ptr must rise from 0 to m and col must lie in [0, n)");

    // CSR-in: counts into in_ptr[1..n], exclusive scan, scatter with a cursor
    int32_t *cnt = nullptr;
    st = alloc_buf(ix, (void **)&cnt, sizeof(int32_t) * ((size_t)n + 1), s);
    if (st) return st;
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), s);
    if (m) { k_count_in<<<grid_for(m), kBlock, 0, s>>>(ix->out_col, m, cnt); ++ix->launches; }
    st = exclusive_scan_i32(ix, cnt, ix->in_ptr, (int64_t)n + 1, s);
    if (st) { free_buf(ix, cnt, s); return st; }
    cudaMemcpyAsync(cnt, ix->in_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s);
    if (m) {
        const int64_t hcap = m / kHeavyDeg + 1;  // rows of kHeavyDeg edges or more
        int32_t *heavy = nullptr;
        if ((st = alloc_buf(ix, (void **)&heavy, sizeof(int32_t) * ((size_t)hcap + 1), s))) {
            free_buf(ix, cnt, s);
            return st;
        }
        uint32_t *nheavy = reinterpret_cast<uint32_t *>(heavy + hcap);
        cudaMemsetAsync(nheavy, 0, sizeof(uint32_t), s);
        k_scatter_in<<<grid_for((int64_t)n), kBlock, 0, s>>>(ix->out_ptr, ix->out_col, n, cnt, ix->in_col, heavy,
                                                               nheavy);
        k_scatter_in_heavy<<<(unsigned)num_sms() * 2, 1024, 0, s>>>(ix->out_ptr, ix->out_col, cnt, ix->in_col, heavy,
                                                                     nheavy);
        ix->launches += 2;
        free_buf(ix, heavy, s);
    }
    free_buf(ix, cnt, s);
    k_fill_vmeta<<<grid_for(n), kBlock, 0, s>>>(ix->out_ptr, ix->in_ptr, n, ix->slots0, ix->vm, ix->d_status);
    ++ix->launches;
    e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "prep_graph");
    st = read_status(ix, s);
    if (st) return fail(ix, st, "a vertex has 2^27 or more base edges in one direction");
    return DBL_OK;
}

// ------------------------------------------------------------ landmarks
// The ranking key of a vertex: M(u) = |Suc(u)| * |Pre(u)| from the two CSRs,
// or an explicit 64-bit key array (e.g. learned scores); larger ranks first,
// ties by smaller id.
// rule (without explicit keys): 0 = |Suc| * |Pre| (Section 4.1), and Table
// 3's 1 = max, 2 = min, 3 = sum of the two degrees.
struct KeySrc {
    const int32_t *op, *ip;
    const unsigned long long *keys;
    int rule;
};

__device__ __forceinline__ unsigned long long key_of(const KeySrc &ks, int32_t v)
{
    if (ks.keys) return ks.keys[v];
    unsigned long long o = (unsigned long long)(ks.op[v + 1] - ks.op[v]);
    unsigned long long i = (unsigned long long)(ks.ip[v + 1] - ks.ip[v]);
    switch (ks.rule) {
    case 1: return o > i ? o : i;
    case 2: return o < i ? o : i;
    case 3: return o + i;
    default: return o * i;
    }
}

struct SelState {
    unsigned long long prefix;  // bits of T decided so far
    unsigned long long pmask;   // which bits are decided
    long long need;             // how many more to take inside the current prefix
    long long above;            // vertices strictly above the current prefix range
    unsigned int hist[256];
};

__global__ void k_sel_hist(KeySrc ks, int32_t n, SelState *st, int shift)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long pre = st->prefix, pm = st->pmask;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long M = key_of(ks, (int32_t)v);
        if ((M & pm) == pre) atomicAdd(&h[(M >> shift) & 255], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&st->hist[i], h[i]);
}

__global__ void k_sel_pick(SelState *st, int shift)
{
    if (threadIdx.x != 0) return;
    long long need = st->need;
    int b = 255;
    for (; b > 0; --b) {
        long long c = st->hist[b];
        if (c >= need) break;
        need -= c;
        st->above += c;
    }
    st->need = need;
    st->prefix |= (unsigned long long)b << shift;
    st->pmask |= 255ull << shift;
    for (int i = 0; i < 256; ++i) st->hist[i] = 0;
}

// vertices with M > T (unordered) and flags of M == T
__global__ void k_sel_gather(KeySrc ks, int32_t n, const SelState *st, int32_t *above, uint32_t *n_above,
                             int32_t *tie_flag, int32_t k)
{
    const unsigned long long T = st->prefix;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long M = key_of(ks, (int32_t)v);
        tie_flag[v] = M == T ? 1 : 0;
        if (M > T) {
            uint32_t p = atomicAdd(n_above, 1u);
            if (p < (uint32_t)k) above[p] = (int32_t)v;  // fewer than k lie above the k-th value
        }
    }
}

__global__ void k_sel_ties(const int32_t *tie_flag, const int32_t *tie_rank, int32_t n, const SelState *st,
                           const uint32_t *n_above, int32_t *landmarks, int32_t k)
{
    const long long need = st->need;
    const uint32_t na = *n_above;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (tie_flag[v] && tie_rank[v] < need && (int64_t)na + tie_rank[v] < k)
            landmarks[na + tie_rank[v]] = (int32_t)v;
}

// rank the (< k) vertices above T by (M desc, id asc); one block
__global__ void k_sel_rank(KeySrc ks, const int32_t *above, const uint32_t *n_above, int32_t *landmarks, int32_t k)
{
    const uint32_t na = min(*n_above, (uint32_t)k);
    for (uint32_t i = threadIdx.x; i < na; i += blockDim.x) {
        int32_t a = above[i];
        unsigned long long Ma = key_of(ks, a);
        uint32_t r = 0;
        for (uint32_t j = 0; j < na; ++j) {
            int32_t b = above[j];
            unsigned long long Mb = key_of(ks, b);
            r += (Mb > Ma) || (Mb == Ma && b < a);
        }
        if (r < (uint32_t)k) landmarks[r] = a;
    }
}

__global__ void k_copy_landmarks(const int32_t *user, int32_t k, int32_t n, int32_t *lm, uint32_t *status)
{
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        int32_t l = user[i];
        if (l >= n || l < -1) set_status(status, DBL_ERR_INVALID);
        lm[i] = l < 0 ? -1 : l;
    }
}

dbl_status select_landmarks(dbl_index *ix, const int32_t *user, cudaStream_t s)
{
    const int32_t n = ix->n, k = ix->k;
    if (user) {
        k_copy_landmarks<<<1, kBlock, 0, s>>>(user, k, n, ix->landmarks, ix->d_status);
        ++ix->launches;
        dbl_status st = read_status(ix, s);
        return st ? fail(ix, st, "landmark id out of range") : DBL_OK;
    }
    return select_top(ix, ix->out_ptr, ix->in_ptr, nullptr, n, k, ix->landmarks, s);
}

// out[0..k): the top min(k, n) vertices by key (descending), ties by id; -1 after.
dbl_status select_top(dbl_index *ix, const int32_t *op, const int32_t *ip, const unsigned long long *keys, int32_t n,
                      int32_t k, int32_t *out, cudaStream_t s)
{
    const KeySrc ks{op, ip, keys, ix->opt.landmark_rule};
    cudaMemsetAsync(out, 0xff, sizeof(int32_t) * (size_t)k, s);  // -1
    const int64_t take = k < n ? k : n;
    if (take == 0) return DBL_OK;
    SelState *sel = nullptr;
    int32_t *above = nullptr, *flag = nullptr, *rank = nullptr;
    uint32_t *na = nullptr;
    dbl_status st;
    if ((st = alloc_buf(ix, (void **)&sel, sizeof(SelState), s))) return st;
    if ((st = alloc_buf(ix, (void **)&above, sizeof(int32_t) * (size_t)k + 16, s))) return st;
    if ((st = alloc_buf(ix, (void **)&flag, sizeof(int32_t) * ((size_t)n + 1), s))) return st;
    if ((st = alloc_buf(ix, (void **)&rank, sizeof(int32_t) * ((size_t)n + 1), s))) return st;
    if ((st = alloc_buf(ix, (void **)&na, 16, s))) return st;
    cudaMemsetAsync(sel, 0, sizeof(SelState), s);
    cudaMemsetAsync(na, 0, 16, s);
    // need = take
    long long h_need = take;
    cudaMemcpyAsync(&sel->need, &h_need, sizeof(long long), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);  // h_need is a stack value
    const unsigned grid = grid_for(n);
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_sel_hist<<<grid, kBlock, 0, s>>>(ks, n, sel, shift);
        ++ix->launches;
        k_sel_pick<<<1, 32, 0, s>>>(sel, shift);
        ++ix->launches;
    }
    k_sel_gather<<<grid, kBlock, 0, s>>>(ks, n, sel, above, na, flag, k);
    ++ix->launches;
    st = exclusive_scan_i32(ix, flag, rank, n, s);
    if (!st) {
        k_sel_rank<<<1, kBlock, 0, s>>>(ks, above, na, out, k);
        ++ix->launches;
        k_sel_ties<<<grid, kBlock, 0, s>>>(flag, rank, n, sel, na, out, k);
        ++ix->launches;
    }
    free_buf(ix, sel, s);
    free_buf(ix, above, s);
    free_buf(ix, flag, s);
    free_buf(ix, rank, s);
    free_buf(ix, na, s);
    cudaError_t e = cudaGetLastError();
    return st ? st : (e ? cuda_fail(ix, e, "select_landmarks") : DBL_OK);
}

// ------------------------------------------------------------ leaves
__device__ __forceinline__ int32_t fib_bucket(int32_t v, int32_t kp)
{
    unsigned long long x = (unsigned long long)(uint32_t)v * 0x9E3779B97F4A7C15ull;
    return (int32_t)__umul64hi(x, (unsigned long long)kp);
}

// Leaves from the degrees: zero in-degree seeds BL_in, zero out-degree seeds
// BL_out (Definition 2); with r > 0 also every v with 0 < M(v) <= r, seeding
// both (Section 6, "Label Node Selection").
__global__ void k_leaves_degree(const int32_t *op, const int32_t *ip, int32_t n, int32_t kp, long long r,
                                int32_t *bucket, uint8_t *role)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const long long din = ip[v + 1] - ip[v], dout = op[v + 1] - op[v];
        uint8_t ro = (uint8_t)((din == 0 ? 1 : 0) | (dout == 0 ? 2 : 0));
        if (!ro && din * dout <= r) ro = 3;
        role[v] = ro;
        bucket[v] = ro ? fib_bucket((int32_t)v, kp) : -1;
    }
}

__global__ void k_leaves_user(const int32_t *ub, const uint8_t *ur, int32_t n, int32_t kp, int32_t *bucket,
                              uint8_t *role, uint32_t *status)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = ub[v];
        if (b >= kp || b < -1) set_status(status, DBL_ERR_INVALID);
        uint8_t r = (b >= 0 && b < kp) ? (uint8_t)(ur[v] & 3) : 0;
        role[v] = r;
        bucket[v] = r ? b : -1;
    }
}

dbl_status select_leaves(dbl_index *ix, const int32_t *bucket, const uint8_t *role, cudaStream_t s)
{
    const unsigned grid = grid_for(ix->n);
    if (!bucket) {
        k_leaves_degree<<<grid, kBlock, 0, s>>>(ix->out_ptr, ix->in_ptr, ix->n, ix->kp, (long long)ix->opt.leaf_r,
                                                ix->leaf_bucket, ix->leaf_role);
        ++ix->launches;
        cudaError_t e = cudaGetLastError();
        return e ? cuda_fail(ix, e, "select_leaves") : DBL_OK;
    }
    k_leaves_user<<<grid, kBlock, 0, s>>>(bucket, role, ix->n, ix->kp, ix->leaf_bucket, ix->leaf_role, ix->d_status);
    ++ix->launches;
    dbl_status st = read_status(ix, s);
    return st ? fail(ix, st, "leaf bucket out of range") : DBL_OK;
}

// ------------------------------------------------------------ seeding
__global__ void k_seed_landmarks(const int32_t *lm, int32_t k, uint64_t *rec, int32_t rw, int32_t hs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        int32_t l = lm[i];
        if (l < 0) continue;
        unsigned long long bit = 1ull << (i & 63);
        uint64_t *r = rec + (size_t)l * rw;
        atomicOr((unsigned long long *)(r + (i >> 6)), bit);        // DL_in(l)
        atomicOr((unsigned long long *)(r + hs + (i >> 6)), bit);   // DL_out(l)
    }
}

// bucket b of the BL label is bit bl_base + b of a half (bl_base = 64 * WD,
// or k in the packed layout)
__global__ void k_seed_leaves(const int32_t *bucket, const uint8_t *role, int32_t n, uint64_t *rec, int32_t rw,
                              int32_t hs, int32_t bl_base)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        uint8_t r = role[v];
        if (!r) continue;
        const int32_t pos = bl_base + bucket[v];
        unsigned long long bit = 1ull << (pos & 63);
        uint64_t *p = rec + (size_t)v * rw;
        if (r & 1) p[pos >> 6] |= bit;          // BL_in(v)
        if (r & 2) p[hs + (pos >> 6)] |= bit;   // BL_out(v)
    }
}

// every vertex with a non-zero half joins the frontier in that direction
// (directions in `dirs`: bit 0 forward, bit 1 backward); the halves are read
// through the propagation's record view and the adjacency from its graph.
// With `renum` (the build's renumbering, old id -> new id) the vertices are
// visited in the order of their original ids, so the frontier starts in the
// same order as the propagation in id order would: the level-synchronous
// schedule, and with it how often a vertex is pushed again, stays that of the
// original numbering.
__global__ void k_seed_frontier(RecView rw, int32_t hs, DevGraph g, FrontierOut f, int dirs, const int32_t *renum)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool act = i < g.n;
        const int32_t v = act ? (renum ? renum[i] : (int32_t)i) : 0;
        bool fw = false, bw = false;
        if (act) {
            uint64_t a = 0, b = 0;
            if (dirs & 1) {
                const uint64_t *p = rec_half(rw, v, 0);
                for (int w = 0; w < hs; ++w) a |= p[w];
            }
            if (dirs & 2) {
                const uint64_t *p = rec_half(rw, v, 1);
                for (int w = 0; w < hs; ++w) b |= p[w];
            }
            fw = a != 0;
            bw = b != 0;
        }
        warp_enqueue(fw, v, 0, g, f);
        warp_enqueue(bw, v, 1, g, f);
    }
}

void launch_seed_frontier(dbl_index *ix, cudaStream_t s, int dirs, const int32_t *renum)
{
    FrontierOut f{ix->front[0], ix->d_counts + kCntFront0, ix->front_cap, mark_of(ix, 0), ix->wpd, ix->d_status};
    cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
    int64_t blocks = ((int64_t)ix->n + kBlock - 1) / kBlock;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    k_seed_frontier<<<(unsigned)blocks, kBlock, 0, s>>>(rec_view(ix), ix->hs, prop_graph(ix), f, dirs, renum);
    ++ix->launches;
}

// ------------------------------------------------------------ build order
// The build may propagate over a renumbered copy of the graph in which
// vertices come in groups of equal floor(log2(in-degree + out-degree)), the
// highest group first and ids ascending inside a group (degree-based grouping:
// Faldu, Diamond and Grot, "A Closer Look at Lightweight Graph Reordering",
// IISWC 2019).  On a power-law graph most edges end at the few vertices of the
// top groups (on the 2^24-vertex R-MAT graph the top 10% of vertices hold 92%
// of the edge endpoints); ordered, their records share cache lines and pages,
// where in id order every random record read of the propagation may touch a
// page of its own.  The least fixpoint does not depend on the numbering:
// labels are copied into the new order before and back after.
constexpr int kOrderTile = 1024;  // vertex ids per block of the ordering kernels
constexpr int kOrderSlots = 32;   // degree groups; slot 0 holds the largest degrees
constexpr int kHeavySlots = 21;   // slots 0..20: in + out degree >= 1024 (kHeavyDeg), a block per row

__device__ __forceinline__ int order_slot(int32_t d)
{
    return 31 - (d > 0 ? 32 - __clz(d) : 0);  // degree d in [2^(g-1), 2^g) -> group g, slot 31 - g
}

__device__ __forceinline__ int32_t base_deg(const DevGraph &g, int dir, int32_t x)
{
    return va_deg(load_vadj(g.vm, dir, x).dc);
}

// cnt[slot * ntiles + tile]: vertices of the tile in the slot
__global__ void __launch_bounds__(kOrderTile) k_order_count(DevGraph g, int64_t ntiles, int32_t *cnt)
{
    __shared__ int32_t c[kOrderSlots];
    if (threadIdx.x < kOrderSlots) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kOrderTile + threadIdx.x;
    if (v < g.n) atomicAdd(&c[order_slot(base_deg(g, 0, (int32_t)v) + base_deg(g, 1, (int32_t)v))], 1);
    __syncthreads();
    if (threadIdx.x < kOrderSlots) cnt[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// new id of v = offs[slot, tile] (exclusive scan of cnt, slot-major) + the
// vertices of the same slot before v in its tile; pi: old -> new, sigma: new ->
// old, and v's base degrees at its new place: deg[nv] out, deg[n + 1 + nv] in
__global__ void __launch_bounds__(kOrderTile) k_order_assign(DevGraph g, int64_t ntiles, const int32_t *offs,
                                                              int32_t *pi, int32_t *sigma, int32_t *deg)
{
    __shared__ int32_t w_at[kOrderTile / 32][kOrderSlots];  // per warp and slot: count, then offset in the tile
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    w_at[warp][lane] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kOrderTile + threadIdx.x;
    const bool act = v < g.n;
    const int32_t dout = act ? base_deg(g, 0, (int32_t)v) : 0, din = act ? base_deg(g, 1, (int32_t)v) : 0;
    const int slot = act ? order_slot(dout + din) : kOrderSlots;
    const unsigned peers = __match_any_sync(kFull, slot);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (act && rank == 0) w_at[warp][slot] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < kOrderSlots) {
        int32_t acc = 0;
        for (int w = 0; w < kOrderTile / 32; ++w) {
            const int32_t c = w_at[w][threadIdx.x];
            w_at[w][threadIdx.x] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (act) {
        const int32_t nv = offs[(int64_t)slot * ntiles + blockIdx.x] + w_at[warp][slot] + rank;
        pi[v] = nv;
        sigma[nv] = (int32_t)v;
        deg[nv] = dout;
        deg[(int64_t)g.n + 1 + nv] = din;
    }
}

// metadata of the new order: rows at the scanned offsets, no inserted edges
__global__ void k_order_vmeta(int32_t n, const int32_t *deg, const int32_t *start, VMeta *vm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        VMeta m;
        for (int dir = 0; dir < 2; ++dir) {
            const int64_t j = (int64_t)dir * (n + 1) + i;
            m.d[dir] = VAdj{start[j], va_dc(deg[j], 0), 0, 0};
        }
        vm[i] = m;
    }
}

// row i of the new order = row sigma[i] of the old one, every id renumbered:
// the rows of the heavy slots (new ids below *heavy) a block each ...
__global__ void k_order_rows_heavy(DevGraph g, const int32_t *pi, const int32_t *sigma, const int32_t *heavy,
                                   DevGraph h)
{
    constexpr int U = kWalkUnroll;
    const int64_t hi = *heavy;
    for (int64_t i = blockIdx.x; i < hi; i += gridDim.x) {
        const VMeta src = g.vm[sigma[i]], dst = h.vm[i];
        for (int dir = 0; dir < 2; ++dir) {
            const int32_t *sc = dir ? g.in_col : g.out_col;
            int32_t *dc = const_cast<int32_t *>(dir ? h.in_col : h.out_col);
            const int32_t s0 = src.d[dir].start, d0 = dst.d[dir].start, deg = va_deg(src.d[dir].dc);
            for (int32_t j0 = threadIdx.x; j0 < deg; j0 += U * (int32_t)blockDim.x) {
                int32_t v[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int32_t j = j0 + k * (int32_t)blockDim.x;
                    v[k] = j < deg ? sc[s0 + j] : 0;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) v[k] = pi[v[k]];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int32_t j = j0 + k * (int32_t)blockDim.x;
                    if (j < deg) dc[d0 + j] = v[k];
                }
            }
        }
    }
}

// ... and the others by warps, 32 consecutive new rows at a time, whose
// destinations are one contiguous range per direction
__global__ void k_order_rows_light(DevGraph g, const int32_t *pi, const int32_t *sigma, const int32_t *heavy,
                                   DevGraph h)
{
    constexpr int U = kWalkUnroll;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = *heavy + w * 32; r0 < g.n; r0 += nw * 32) {  // warp-uniform
        const int64_t i = r0 + lane;
        VMeta src{}, dst{};
        if (i < g.n) {
            src = g.vm[sigma[i]];
            dst = h.vm[i];
        }
        for (int dir = 0; dir < 2; ++dir) {
            const int32_t *sc = dir ? g.in_col : g.out_col;
            int32_t *dc = const_cast<int32_t *>(dir ? h.in_col : h.out_col);
            const int32_t d0 = __shfl_sync(kFull, dst.d[dir].start, 0);
            const int32_t b = src.d[dir].start, d = i < g.n ? va_deg(src.d[dir].dc) : 0;
            uint32_t total;
            const uint32_t excl = walk_prefix(d, total);
            for (uint32_t base = 0; base < total; base += 32u * U) {
                int owner[U];
                int32_t p[U], v[U];
                bool ok[U];
                walk_step<U>(excl, b, base, total, owner, p, ok);
#pragma unroll
                for (int k = 0; k < U; ++k) v[k] = ok[k] ? sc[p[k]] : 0;
#pragma unroll
                for (int k = 0; k < U; ++k) v[k] = pi[v[k]];
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (ok[k]) dc[d0 + (int32_t)(base + 32u * k + lane)] = v[k];
            }
        }
    }
}

// dst[r * dst_stride + dst_off + w] = src[idx(r) * src_stride + src_off + w]
// for rows r < n and words w < W; idx(r) = idx[r], or r without idx
__global__ void k_gather_words(const uint64_t *src, int64_t src_stride, int64_t src_off, const int32_t *idx,
                               uint64_t *dst, int64_t dst_stride, int64_t dst_off, int64_t n, int W)
{
    const int64_t words = n * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / W, w = i % W;
        const int64_t sr = idx ? idx[r] : r;
        dst[r * dst_stride + dst_off + w] = src[sr * src_stride + src_off + w];
    }
}

// Buffers of the degree-ordered graph: pi (old -> new), sigma (new -> old),
// its metadata and both adjacency arrays.
struct BuildOrder {
    int32_t *pi = nullptr, *sigma = nullptr, *col = nullptr;
    VMeta *vm = nullptr;
    DevGraph g{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

static void free_order(dbl_index *ix, BuildOrder &bo, cudaStream_t s)
{
    free_buf(ix, bo.pi, s);
    free_buf(ix, bo.sigma, s);
    free_buf(ix, bo.col, s);
    free_buf(ix, bo.vm, s);
    bo = BuildOrder{};
}

// The degree-ordered copy of the index's base graph (the build runs before
// any insertion, so the base edges are all the edges).
static dbl_status make_order(dbl_index *ix, BuildOrder &bo, cudaStream_t s)
{
    const int32_t n = ix->n;
    const int64_t m = ix->m;
    const int64_t ntiles = ((int64_t)n + kOrderTile - 1) / kOrderTile;
    const int64_t ncnt = kOrderSlots * ntiles;
    int32_t *work = nullptr;  // cnt | offs | deg (2 x (n + 1)) | start (2 x (n + 1)) | heavy rows
    const size_t work_words = 2 * (size_t)ncnt + 4 * ((size_t)n + 1) + 1;
    dbl_status st;
    if ((st = alloc_buf(ix, (void **)&bo.pi, sizeof(int32_t) * (size_t)n, s)) ||
        (st = alloc_buf(ix, (void **)&bo.sigma, sizeof(int32_t) * (size_t)n, s)) ||
        (st = alloc_buf(ix, (void **)&bo.vm, sizeof(VMeta) * (size_t)n, s)) ||
        (st = alloc_buf(ix, (void **)&bo.col, sizeof(int32_t) * (2 * (size_t)m + 1), s)) ||
        (st = alloc_buf(ix, (void **)&work, sizeof(int32_t) * work_words, s))) {
        free_buf(ix, work, s);
        free_order(ix, bo, s);
        return st;
    }
    const DevGraph g = dev_graph(ix);
    int32_t *cnt = work, *offs = work + ncnt, *deg = offs + ncnt, *start = deg + 2 * ((int64_t)n + 1);
    int32_t *heavy = start + 2 * ((int64_t)n + 1);
    k_order_count<<<(unsigned)ntiles, kOrderTile, 0, s>>>(g, ntiles, cnt);
    ++ix->launches;
    if ((st = exclusive_scan_i32(ix, cnt, offs, ncnt, s))) {
        free_buf(ix, work, s);
        free_order(ix, bo, s);
        return st;
    }
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * 2 * ((size_t)n + 1), s);
    k_order_assign<<<(unsigned)ntiles, kOrderTile, 0, s>>>(g, ntiles, offs, bo.pi, bo.sigma, deg);
    ++ix->launches;
    // vertices of the heavy slots: the offset of the first light slot
    cudaMemcpyAsync(heavy, offs + (int64_t)kHeavySlots * ntiles, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    // one scan over both directions: the in-rows start after the m out-edges
    if ((st = exclusive_scan_i32(ix, deg, start, 2 * ((int64_t)n + 1), s))) {
        free_buf(ix, work, s);
        free_order(ix, bo, s);
        return st;
    }
    k_order_vmeta<<<grid_for(n), kBlock, 0, s>>>(n, deg, start, bo.vm);
    ++ix->launches;
    bo.g = DevGraph{n, bo.vm, bo.col, bo.col, nullptr, nullptr, nullptr};
    k_order_rows_heavy<<<(unsigned)num_sms() * 2, 1024, 0, s>>>(g, bo.pi, bo.sigma, heavy, bo.g);
    k_order_rows_light<<<grid_for(n), kBlock, 0, s>>>(g, bo.pi, bo.sigma, heavy, bo.g);
    ix->launches += 2;
    free_buf(ix, work, s);
    cudaError_t e = cudaGetLastError();
    if (e) {
        free_order(ix, bo, s);
        return cuda_fail(ix, e, "build order");
    }
    return DBL_OK;
}

// The build's propagation to the least fixpoint from the seeded records.
// When the records are larger than the address-translation caches cover
// (random 32-byte gathers drop from ~70 G/s over 256 MB to ~30 G/s over
// 512 MB on GB300), the two directions are propagated one after the other,
// each over an array of that direction's halves alone (half the bytes
// touched at random), and interleaved back into the records at the end; and
// the propagation runs over the degree-ordered copy of the graph (above).
// All forms give the same least fixpoint: the directions never read each
// other, and the numbering changes only where a record is stored.
constexpr size_t kSplitBuildBytes = 256ull << 20;

dbl_status build_propagate(dbl_index *ix, cudaStream_t s)
{
    const size_t rec_bytes = sizeof(uint64_t) * (size_t)ix->n * ix->rw;
    const bool big = rec_bytes > kSplitBuildBytes;
    const bool split = ix->opt.build_split > 0 || (ix->opt.build_split == 0 && big);
    // (the ordered copy keeps both directions' rows in one int32-indexed array)
    const bool order = ix->n > 0 && 2 * ix->m < (1ll << 31) &&
                       (ix->opt.build_order > 0 || (ix->opt.build_order == 0 && big));
    if (!split && !order) {
        launch_seed_frontier(ix, s, 3);
        return propagate(ix, s);
    }
    const int64_t n = ix->n, hs = ix->hs, rw = ix->rw;
    const int parts = split ? 2 : 1;
    uint64_t *arr[2] = {nullptr, nullptr};
    BuildOrder bo;
    dbl_status st;
    if (order) {  // the renumbered graph counts as graph preparation
        tbegin(ix, DBL_KERNEL_BUILD_PREP, s);
        st = make_order(ix, bo, s);
        tend(ix, s);
        if (st) return st;
    }
    tbegin(ix, DBL_KERNEL_PROPAGATE, s);  // the copies count as the build's propagation
    for (int d = 0; d < parts; ++d)
        if ((st = alloc_buf(ix, (void **)&arr[d], split ? rec_bytes / 2 : rec_bytes, s))) {
            tend(ix, s);
            free_buf(ix, arr[0], s);
            free_order(ix, bo, s);
            return st;
        }
    const unsigned grid = grid_for(n * (split ? hs : rw));
    for (int d = 0; d < parts; ++d) {  // halves (or records) into the propagation's order
        if (split) k_gather_words<<<grid, kBlock, 0, s>>>(ix->rec, rw, d * hs, bo.sigma, arr[d], hs, 0, n, (int)hs);
        else k_gather_words<<<grid, kBlock, 0, s>>>(ix->rec, rw, 0, bo.sigma, arr[0], rw, 0, n, (int)rw);
        ++ix->launches;
    }
    tend(ix, s);
    ix->prop_graph = bo.g;
    st = DBL_OK;
    for (int d = 0; d < parts && !st; ++d) {
        ix->prop_view = split ? RecView{arr[d], hs, 0} : RecView{arr[0], rw, hs};
        launch_seed_frontier(ix, s, split ? 1 << d : 3, bo.pi);
        st = propagate(ix, s);
    }
    ix->prop_view = RecView{nullptr, 0, 0};
    ix->prop_graph = DevGraph{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (!st) {
        tbegin(ix, DBL_KERNEL_PROPAGATE, s);
        for (int d = 0; d < parts; ++d) {  // and back into the records, in id order
            if (split) k_gather_words<<<grid, kBlock, 0, s>>>(arr[d], hs, 0, bo.pi, ix->rec, rw, d * hs, n, (int)hs);
            else k_gather_words<<<grid, kBlock, 0, s>>>(arr[0], rw, 0, bo.pi, ix->rec, rw, 0, n, (int)rw);
            ++ix->launches;
        }
        tend(ix, s);
    }
    free_buf(ix, arr[0], s);
    free_buf(ix, arr[1], s);
    free_order(ix, bo, s);
    cudaError_t e = cudaGetLastError();
    if (!st && e) st = cuda_fail(ix, e, "build propagation");
    return st;
}

dbl_status seed_labels(dbl_index *ix, cudaStream_t s)
{
    cudaMemsetAsync(ix->rec, 0, sizeof(uint64_t) * (size_t)ix->n * ix->rw, s);
    k_seed_landmarks<<<1, kBlock, 0, s>>>(ix->landmarks, ix->k, ix->rec, ix->rw, ix->hs);
    ++ix->launches;
    k_seed_leaves<<<grid_for(ix->n), kBlock, 0, s>>>(ix->leaf_bucket, ix->leaf_role, ix->n, ix->rec, ix->rw, ix->hs,
                                                      ix->bl_base);
    ++ix->launches;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(ix, e, "seed_labels") : DBL_OK;
}

}  // namespace dbl
