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

// scatter u into Pre(col[e]) for every edge u -> col[e] (one warp per source row)
__global__ void k_scatter_in(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t *cursor,
                             int32_t *in_col)
{
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w; u < n; u += nw) {
        int32_t b = row_ptr[u], e = row_ptr[u + 1];
        for (int32_t j = b + lane; j < e; j += 32) {
            int32_t v = col[j];
            int32_t pos = atomicAdd(cursor + v, 1);
            in_col[pos] = (int32_t)u;
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
    if (m) { k_scatter_in<<<grid_for((int64_t)n * 32), kBlock, 0, s>>>(ix->out_ptr, ix->out_col, n, cnt, ix->in_col); ++ix->launches; }
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
// (directions in `dirs`: bit 0 forward, bit 1 backward)
__global__ void k_seed_frontier(const uint64_t *rec, int32_t rw, int32_t hs, DevGraph g, FrontierOut f, int dirs)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += stride) {
        int64_t v = base + threadIdx.x;
        bool act = v < g.n;
        bool fw = false, bw = false;
        if (act) {
            const uint64_t *p = rec + (size_t)v * rw;
            uint64_t a = 0, b = 0;
            for (int i = 0; i < hs; ++i) {
                a |= p[i];
                b |= p[hs + i];
            }
            fw = (dirs & 1) && a != 0;
            bw = (dirs & 2) && b != 0;
        }
        warp_enqueue(fw, (int32_t)v, 0, g, f);
        warp_enqueue(bw, (int32_t)v, 1, g, f);
    }
}

void launch_seed_frontier(dbl_index *ix, cudaStream_t s, int dirs)
{
    FrontierOut f{ix->front[0], ix->d_counts + kCntFront0, ix->front_cap, mark_of(ix, 0), ix->wpd, ix->d_status};
    cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
    int64_t blocks = ((int64_t)ix->n + kBlock - 1) / kBlock;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    k_seed_frontier<<<(unsigned)blocks, kBlock, 0, s>>>(ix->rec, ix->rw, ix->hs, dev_graph(ix), f, dirs);
    ++ix->launches;
}

// The build's propagation to the least fixpoint from the seeded records.
// When the records are larger than the address-translation caches cover
// (random 32-byte gathers drop from ~70 G/s over 256 MB to ~30 G/s over
// 512 MB on GB300), the two directions are propagated one after the other,
// each over an array of that direction's halves alone (half the bytes
// touched at random), and interleaved back into the records at the end.
// Both give the same least fixpoint: the directions never read each other.
constexpr size_t kSplitBuildBytes = 256ull << 20;

__global__ void k_split_halves(const uint64_t *rec, int64_t n, int hs, uint64_t *fw, uint64_t *bw)
{
    const int64_t words = n * hs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i / hs, w = i % hs;
        fw[i] = rec[x * 2 * hs + w];
        bw[i] = rec[x * 2 * hs + hs + w];
    }
}

__global__ void k_join_halves(uint64_t *rec, int64_t n, int hs, const uint64_t *fw, const uint64_t *bw)
{
    const int64_t words = n * hs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i / hs, w = i % hs;
        rec[x * 2 * hs + w] = fw[i];
        rec[x * 2 * hs + hs + w] = bw[i];
    }
}

dbl_status build_propagate(dbl_index *ix, cudaStream_t s)
{
    const size_t rec_bytes = sizeof(uint64_t) * (size_t)ix->n * ix->rw;
    const bool split = ix->opt.build_split > 0 || (ix->opt.build_split == 0 && rec_bytes > kSplitBuildBytes);
    if (!split) {
        launch_seed_frontier(ix, s, 3);
        return propagate(ix, s);
    }
    uint64_t *half[2] = {nullptr, nullptr};
    dbl_status st;
    for (int d = 0; d < 2; ++d)
        if ((st = alloc_buf(ix, (void **)&half[d], rec_bytes / 2, s))) {
            free_buf(ix, half[0], s);
            return st;
        }
    const unsigned grid = grid_for((int64_t)ix->n * ix->hs);
    tbegin(ix, DBL_KERNEL_PROPAGATE, s);  // the copies count as the build's propagation
    k_split_halves<<<grid, kBlock, 0, s>>>(ix->rec, ix->n, ix->hs, half[0], half[1]);
    ++ix->launches;
    tend(ix, s);
    st = DBL_OK;
    for (int d = 0; d < 2 && !st; ++d) {
        launch_seed_frontier(ix, s, 1 << d);
        ix->prop_view = RecView{half[d], (int64_t)ix->hs, 0};
        st = propagate(ix, s);
        ix->prop_view = RecView{nullptr, 0, 0};
    }
    if (!st) {
        tbegin(ix, DBL_KERNEL_PROPAGATE, s);
        k_join_halves<<<grid, kBlock, 0, s>>>(ix->rec, ix->n, ix->hs, half[0], half[1]);
        ++ix->launches;
        tend(ix, s);
    }
    free_buf(ix, half[0], s);
    free_buf(ix, half[1], s);
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
