// Learned landmark scorer (not in the paper; the paper ranks landmarks by
// M(u) = |Pre(u)| * |Suc(u)|, Section 4.1, and notes that the best choice is
// NP-hard).  A 16-128-128-1 ReLU network scores every vertex from 16
// log-scaled counts; it is trained on how many sampled reachable pairs each
// vertex would decide as a landmark.  Answers stay exact for any ranking:
// only which pairs the DL test decides changes.
//
//   features   per-vertex counts -> bf16 [n][16]            (one warp per vertex)
//   coverage   count[c] = #{j : u_j reaches c, c reaches v_j} for sampled pairs,
//              256 pairs per pass as bits of a 4-word record, propagated with the
//              same frontier kernels as the labels
//   MLP        bf16 operands, fp32 accumulate on the 5th-generation tensor
//              cores (tcgen05.mma, accumulators in TMEM, read back with
//              tcgen05.ld): a fused forward over 128-row tiles fed by TMA, and
//              a backward of three 128 x 128-tile GEMMs with split-K reductions
//   selection  top-k by score with the landmark radix select
#include <cuda_bf16.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
#include "dbl_tc.cuh"
#include "dbl_kernels.cuh"

namespace dbl {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ features
__device__ __forceinline__ int32_t indeg_of(const DevGraph &g, int32_t x) { return deg_of(g, 1, x); }
__device__ __forceinline__ int32_t outdeg_of(const DevGraph &g, int32_t x) { return deg_of(g, 0, x); }

__global__ void k_mark_landmarks(const int32_t *lm, int32_t k, uint8_t *mark)
{
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        if (lm[i] >= 0) mark[lm[i]] = 1;
}

// One warp per vertex; lanes stride over Pre and Suc for the neighbour sums.
__global__ void k_features(DevGraph g, const uint64_t *rec, int32_t hs, int32_t wd, int32_t wb, int packed,
                           uint64_t dlm, const uint8_t *mark, bf16 *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t xv = w0; xv < g.n; xv += nw) {
        const int32_t x = (int32_t)xv;
        unsigned long long s[6] = {0, 0, 0, 0, 0, 0};  // pre_indeg, suc_outdeg, pre_outdeg, suc_indeg, pre_src, suc_sink
        for (int dir = 0; dir < 2; ++dir) {
            const AdjRange r = adj_of(g, dir, x);
            for (int32_t e = lane; e < r.bd + r.od; e += 32) {
                const int32_t y = adj_at(g, dir, r, e);
                const unsigned long long di = (unsigned long long)indeg_of(g, y);
                const unsigned long long dout = (unsigned long long)outdeg_of(g, y);
                if (dir == 1) {          // y in Pre(x)
                    s[0] += di;
                    s[2] += dout;
                    s[4] += di == 0;
                } else {                 // y in Suc(x)
                    s[1] += dout;
                    s[3] += di;
                    s[5] += dout == 0;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int o = 16; o; o >>= 1) s[i] += __shfl_xor_sync(kFull, s[i], o);
        if (lane < 16) {
            const uint64_t *p = rec + (size_t)x * 2 * hs;
            double v = 0;
            const double din = (double)indeg_of(g, x), dout = (double)outdeg_of(g, x);
            int pc[4] = {0, 0, 0, 0};
            if (packed) {  // one word per half: DL bits dlm, BL the bits above
                pc[0] = __popcll(p[0] & dlm);
                pc[1] = __popcll(p[1] & dlm);
                pc[2] = __popcll(p[0] & ~dlm);
                pc[3] = __popcll(p[1] & ~dlm);
            } else {
                for (int w = 0; w < wd; ++w) {
                    pc[0] += __popcll(p[w]);
                    pc[1] += __popcll(p[hs + w]);
                }
                for (int w = 0; w < wb; ++w) {
                    pc[2] += __popcll(p[wd + w]);
                    pc[3] += __popcll(p[hs + wd + w]);
                }
            }
            switch (lane) {
            case 0: v = din; break;
            case 1: v = dout; break;
            case 2: v = din * dout; break;
            case 3: v = din + dout; break;
            case 4: v = (double)s[0]; break;
            case 5: v = (double)s[1]; break;
            case 6: v = (double)s[2]; break;
            case 7: v = (double)s[3]; break;
            case 8: v = pc[0]; break;
            case 9: v = pc[1]; break;
            case 10: v = pc[2]; break;
            case 11: v = pc[3]; break;
            case 12: v = (double)pc[0] * pc[1]; break;
            case 13: v = (double)s[4]; break;
            case 14: v = (double)s[5]; break;
            default: v = mark[x] ? 1.0 : 0.0; break;
            }
            out[(size_t)x * 16 + lane] = __float2bfloat16_rn(log1pf((float)v));
        }
    }
}

dbl_status features(dbl_index *ix, bf16 *out, cudaStream_t s)
{
    uint8_t *mark = nullptr;
    dbl_status st = alloc_buf(ix, (void **)&mark, (size_t)ix->n + 16, s);
    if (st) return st;
    cudaMemsetAsync(mark, 0, (size_t)ix->n + 16, s);
    k_mark_landmarks<<<1, kBlock, 0, s>>>(ix->landmarks, ix->k, mark);
    ++ix->launches;
    int64_t blocks = ((int64_t)ix->n * 32 + kBlock - 1) / kBlock;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    k_features<<<(unsigned)blocks, kBlock, 0, s>>>(dev_graph(ix), ix->rec, ix->hs, ix->wd, ix->wb, ix->packed ? 1 : 0,
                                                   ix->dl_mask, mark, out);
    ++ix->launches;
    free_buf(ix, mark, s);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(ix, e, "features") : DBL_OK;
}

// ------------------------------------------------------------ coverage
constexpr int kCovHS = 4;              // 256 pairs per pass
constexpr int kCovPairs = 64 * kCovHS;

// Keep pair j if it is reachable (reach[j] != 0, or reach == NULL) and the
// first base_slots landmarks do not already decide it (DL_out(u) & DL_in(v)
// restricted to those slots is empty); kept pairs are compacted into (cu, cv).
__global__ void k_cov_filter(const int32_t *u, const int32_t *v, const uint8_t *reach, int64_t pairs, int32_t n,
                             const uint64_t *rec, int32_t hs, int32_t wd, int32_t base_slots, int32_t *cu, int32_t *cv,
                             uint32_t *n_kept, uint32_t *status)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < pairs; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[j], b = v[j];
        if ((uint32_t)a >= (uint32_t)n || (uint32_t)b >= (uint32_t)n) {
            set_status(status, DBL_ERR_INVALID);
            continue;
        }
        if (reach && !reach[j]) continue;
        bool decided = false;
        for (int w = 0; w < wd && w * 64 < base_slots; ++w) {
            const int rem = base_slots - w * 64;
            const uint64_t mask = rem >= 64 ? ~0ull : ((1ull << rem) - 1);
            decided |= (rec[(size_t)a * 2 * hs + hs + w] & rec[(size_t)b * 2 * hs + w] & mask) != 0;
        }
        if (decided) continue;
        const uint32_t p = atomicAdd(n_kept, 1u);
        cu[p] = a;
        cv[p] = b;
    }
}

__global__ void k_cov_seed(const int32_t *u, const int32_t *v, int64_t j0, int64_t j1, int32_t n, uint64_t *crec,
                           DevGraph g, FrontierOut f, uint32_t *status)
{
    for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[j], b = v[j];
        if ((uint32_t)a >= (uint32_t)n || (uint32_t)b >= (uint32_t)n) {
            set_status(status, DBL_ERR_INVALID);
            continue;
        }
        const int bit = (int)(j - j0);
        const unsigned long long m = 1ull << (bit & 63);
        atomicOr((unsigned long long *)(crec + (size_t)a * 2 * kCovHS + (bit >> 6)), m);            // F(u_j)
        atomicOr((unsigned long long *)(crec + (size_t)b * 2 * kCovHS + kCovHS + (bit >> 6)), m);   // B(v_j)
        any_enqueue(a, 0, g, f);
        any_enqueue(b, 1, g, f);
    }
}

__global__ void k_cov_accumulate(const uint64_t *crec, int32_t n, uint32_t *count)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *p = crec + (size_t)x * 2 * kCovHS;
        int c = 0;
#pragma unroll
        for (int w = 0; w < kCovHS; ++w) c += __popcll(p[w] & p[kCovHS + w]);
        if (c) count[x] += (uint32_t)c;
    }
}

__global__ void k_cov_targets(const uint32_t *count, int32_t n, float *t)
{
    __shared__ unsigned int mx;
    // single block: max, then log1p scaling
    if (threadIdx.x == 0) mx = 0;
    __syncthreads();
    unsigned int m = 0;
    for (int64_t x = threadIdx.x; x < n; x += blockDim.x) m = max(m, count[x]);
    atomicMax(&mx, m);
    __syncthreads();
    const float den = mx ? log1pf((float)mx) : 1.0f;
    for (int64_t x = threadIdx.x; x < n; x += blockDim.x) t[x] = log1pf((float)count[x]) / den;
}

dbl_status coverage(dbl_index *ix, const int32_t *u_in, const int32_t *v_in, const uint8_t *reach, int64_t pairs_in,
                    int32_t base_slots, uint32_t *count, int64_t *kept, cudaStream_t s)
{
    uint64_t *crec = nullptr;
    int32_t *cu = nullptr, *cv = nullptr;
    const size_t bytes = sizeof(uint64_t) * (size_t)ix->n * 2 * kCovHS;
    dbl_status st;
    if ((st = alloc_buf(ix, (void **)&crec, bytes, s)) ||
        (st = alloc_buf(ix, (void **)&cu, sizeof(int32_t) * (size_t)pairs_in + 16, s)) ||
        (st = alloc_buf(ix, (void **)&cv, sizeof(int32_t) * (size_t)pairs_in + 16, s)))
        return st;
    cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)ix->n, s);
    cudaMemsetAsync(ix->d_counts + kCntTasks, 0, sizeof(uint32_t), s);
    k_cov_filter<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((pairs_in + kBlock - 1) / kBlock,
                                                                    (int64_t)num_sms() * 16)),
                   kBlock, 0, s>>>(u_in, v_in, reach, pairs_in, ix->n, ix->rec, ix->hs, ix->wd, base_slots, cu, cv,
                                   ix->d_counts + kCntTasks, ix->d_status);
    ++ix->launches;
    cudaMemcpyAsync(ix->h_pinned, ix->d_counts + kCntTasks, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e0 = cudaStreamSynchronize(s);
    if (e0) return cuda_fail(ix, e0, "coverage filter");
    const int64_t pairs = ix->h_pinned[0];
    if (kept) *kept = pairs;
    const int32_t *u = cu, *v = cv;
    for (int64_t j0 = 0; j0 < pairs && !st; j0 += kCovPairs) {
        const int64_t j1 = j0 + kCovPairs < pairs ? j0 + kCovPairs : pairs;
        cudaMemsetAsync(crec, 0, bytes, s);
        FrontierOut f{ix->front[0], ix->d_counts + kCntFront0, ix->front_cap, mark_of(ix, 0), ix->wpd, ix->d_status};
        cudaMemsetAsync(ix->d_counts + kCntFront0, 0, sizeof(uint32_t), s);
        k_cov_seed<<<(unsigned)((j1 - j0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(u, v, j0, j1, ix->n, crec,
                                                                                   dev_graph(ix), f, ix->d_status);
        ++ix->launches;
        st = propagate_records(ix, crec, kCovHS, s);
        if (st) break;
        int64_t blocks = ((int64_t)ix->n + kBlock - 1) / kBlock;
        if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
        k_cov_accumulate<<<(unsigned)(blocks < 1 ? 1 : blocks), kBlock, 0, s>>>(crec, ix->n, count);
        ++ix->launches;
    }
    free_buf(ix, crec, s);
    free_buf(ix, cu, s);
    free_buf(ix, cv, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(ix, e, "coverage") : DBL_OK;
}

// ------------------------------------------------------------ tensor-core kernels
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

constexpr int kH = 128;       // hidden width
constexpr int kF = 16;        // features

// Parameter offsets in the flat fp32 vector (18,817 values).
constexpr int kOffW1 = 0;                     // [16][128]  (in x out)
constexpr int kOffB1 = kOffW1 + kF * kH;      // [128]
constexpr int kOffW2 = kOffB1 + kH;           // [128][128] (in x out)
constexpr int kOffB2 = kOffW2 + kH * kH;      // [128]
constexpr int kOffW3 = kOffB2 + kH;           // [128]
constexpr int kOffB3 = kOffW3 + kH;           // [1]
constexpr int kNumParams = kOffB3 + 1;

// Position of element (row, k) in a [K / 8][rows][8] operand tile (the
// K-block layout of dbl_tc.cuh).
__host__ __device__ constexpr int kblk(int row, int k, int rows) { return (k >> 3) * rows * 8 + row * 8 + (k & 7); }

struct MlpDev {
    const bf16 *W1c;      // layer-1 B operand, N = 128 (out) x K = 16 (in), K-block layout
    const bf16 *W2c;      // layer-2 B operand, N = 128 (out) x K = 128 (in), K-block layout
    const float *p;       // fp32 parameters (biases, w3, b3)
};

constexpr int kTileR = 128;                 // rows per tile: the MMA's M
constexpr uint32_t kWaitLimit = 1u << 22;   // polls of an mbarrier before a kernel gives up

// Shared memory of the forward kernel (operand tiles first, 4 KB aligned).
// The block requests more than it uses: at most two blocks (2 x 256 TMEM
// columns) then share an SM, and every address a tile descriptor can reach,
// even with its two byte offsets exchanged (rows 15 x 2 KB apart), stays
// inside the block's allocation.
struct FwdSmem {
    bf16 x[2][kTileR * kF];
    bf16 w1[kH * kF];
    bf16 h1[kTileR * kH];
    bf16 w2[kH * kH];
    float b1[kH], b2[kH], w3[kH];
    float ypart[kTileR];  // second warpgroup's half of each row's output dot product
    uint64_t bar_w, bar_x[2], bar_mma;
    uint32_t tmem;
};
constexpr int kFwdSmemBytes = 112 * 1024;
constexpr int kFwdThreads = 2 * kTileR;  // two warpgroups: each row's columns split in halves
static_assert(sizeof(FwdSmem) + 1024 <= kFwdSmemBytes, "forward shared memory");
static_assert(offsetof(FwdSmem, w2) + 7 * 4096 + 15 * 2048 + 256 <= kFwdSmemBytes, "descriptor reach");

// Fused forward on the 5th-generation tensor cores.  A block owns 128-row
// tiles: X (128 x 16 bf16) arrives by a TMA tensor copy (or by the threads
// when rows are gathered), layer 1 is one 128 x 128 x 16 MMA into TMEM columns
// [0, 128), the epilogue adds b1, applies ReLU and writes H1 as bf16 back to
// shared memory, layer 2 is eight 128 x 128 x 16 MMAs into columns [128, 256),
// and its epilogue adds b2, applies ReLU, rounds H2 to bf16 and takes the dot
// product with w3.  Two warpgroups: warp w reads TMEM lanes 32 (w % 4) ..
// 32 (w % 4) + 31 (its rows), warpgroup 0 columns 0-63 and warpgroup 1
// columns 64-127 of each layer; the two halves of a row's dot product are
// added through shared memory in a fixed order.  The next tile's X copy is in
// flight during the current tile.  Every wait is bounded:
// on a timeout the block raises *err, waits (bounded) for its copies and MMAs,
// frees its TMEM and returns.
__global__ void __launch_bounds__(kFwdThreads, 1)
    k_mlp_forward(const __grid_constant__ CUtensorMap xmap, int use_tma, MlpDev m, const bf16 *X,
                  const int32_t *rows_idx, int64_t R, float *y, bf16 *H1out, bf16 *H2out, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>(dsm);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        tc::mbar_init(&S.bar_w, 1);
        tc::mbar_init(&S.bar_x[0], 1);
        tc::mbar_init(&S.bar_x[1], 1);
        tc::mbar_init(&S.bar_mma, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, 256);
    for (int i = tid; i < kH; i += blockDim.x) {
        S.b1[i] = m.p[kOffB1 + i];
        S.b2[i] = m.p[kOffB2 + i];
        S.w3[i] = m.p[kOffW3 + i];
    }
    const float b3 = m.p[kOffB3];
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const int row = (warp & 3) * 32 + (tid & 31);  // this thread's row of the tile (TMEM lane)
    const int half = warp >> 2;                    // columns [64 half, 64 half + 64) of each layer
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int64_t ntiles = (R + kTileR - 1) / kTileR;
    bool x_pending[2] = {false, false};  // a tensor copy into x[b] not yet waited for
    if (tid == 0) {
        tc::mbar_expect_tx(&S.bar_w, (uint32_t)(sizeof(S.w1) + sizeof(S.w2)));
        tc::bulk_g2s(S.w1, m.W1c, (uint32_t)sizeof(S.w1), &S.bar_w);
        tc::bulk_g2s(S.w2, m.W2c, (uint32_t)sizeof(S.w2), &S.bar_w);
    }
    if (use_tma && (int64_t)blockIdx.x < ntiles) {
        if (tid == 0) {
            tc::mbar_expect_tx(&S.bar_x[0], (uint32_t)sizeof(S.x[0]));
            tc::tma_load_3d(S.x[0], &xmap, 0, (int32_t)(blockIdx.x * kTileR), 0, &S.bar_x[0]);
        }
        x_pending[0] = true;
    }
    bool ok = __syncthreads_and(tc::mbar_wait(&S.bar_w, 0, kWaitLimit));
    uint32_t px[2] = {0, 0}, pm = 0;
    bool mma_pending = false;
    const uint32_t id = tc::idesc_bf16(kTileR, kH);
    int it = 0;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const int64_t r = tile * kTileR + row;
        if (use_tma) {
            ok = tc::mbar_wait(&S.bar_x[buf], px[buf], kWaitLimit);
            if (ok) {
                px[buf] ^= 1;
                x_pending[buf] = false;
            }
        } else if (half == 0) {
            uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
            if (r < R) {
                const int64_t src = rows_idx ? (int64_t)rows_idx[r] : r;
                const uint4 *xp = reinterpret_cast<const uint4 *>(X + src * kF);
                lo = xp[0];
                hi = xp[1];
            }
            uint4 *xs = reinterpret_cast<uint4 *>(S.x[buf]);
            xs[row] = lo;           // K block 0
            xs[kTileR + row] = hi;  // K block 1
            tc::fence_async_smem();
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        // layer 1; the next tile's X goes into the other buffer, whose last
        // reader (the previous tile's layer-1 MMA) has completed
        const int64_t nxt = tile + gridDim.x;
        if (use_tma && nxt < ntiles) x_pending[buf ^ 1] = true;
        if (tid == 0) {
            if (use_tma && nxt < ntiles) {
                tc::mbar_expect_tx(&S.bar_x[buf ^ 1], (uint32_t)sizeof(S.x[0]));
                tc::tma_load_3d(S.x[buf ^ 1], &xmap, 0, (int32_t)(nxt * kTileR), 0, &S.bar_x[buf ^ 1]);
            }
            tc::tc_fence_after();
            tc::mma_bf16(tmem, tc::smem_desc(S.x[buf], kTileR * 16, 128), tc::smem_desc(S.w1, kH * 16, 128), id, 0u);
            tc::mma_commit(&S.bar_mma);
        }
        mma_pending = true;
        ok = __syncthreads_and(tc::mbar_wait(&S.bar_mma, pm, kWaitLimit));
        if (!ok) break;
        pm ^= 1;
        mma_pending = false;
        tc::tc_fence_after();
        uint4 *h1 = reinterpret_cast<uint4 *>(S.h1);
        float v1[64];  // this thread's 64 columns of layer 1, one TMEM load
        tc::tmem_ld64(tmem + lane_base + (uint32_t)(half * 64), v1);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = half * 4 + cc;
            const float *v = v1 + cc * 16;
            uint32_t pk[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = c * 16 + 2 * j;
                pk[j] = pack_bf16(fmaxf(v[2 * j] + S.b1[col], 0.f), fmaxf(v[2 * j + 1] + S.b1[col + 1], 0.f));
            }
            const uint4 q0 = make_uint4(pk[0], pk[1], pk[2], pk[3]), q1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            h1[(2 * c) * kTileR + row] = q0;
            h1[(2 * c + 1) * kTileR + row] = q1;
            if (H1out && r < R) {
                uint4 *g = reinterpret_cast<uint4 *>(H1out + r * kH + c * 16);
                g[0] = q0;
                g[1] = q1;
            }
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll
            for (int k = 0; k < kH / 16; ++k)
                tc::mma_bf16(tmem + kH, tc::smem_desc(S.h1 + k * 2 * kTileR * 8, kTileR * 16, 128),
                             tc::smem_desc(S.w2 + k * 2 * kH * 8, kH * 16, 128), id, k > 0 ? 1u : 0u);
            tc::mma_commit(&S.bar_mma);
        }
        mma_pending = true;
        ok = __syncthreads_and(tc::mbar_wait(&S.bar_mma, pm, kWaitLimit));
        if (!ok) break;
        pm ^= 1;
        mma_pending = false;
        tc::tc_fence_after();
        float acc = 0.f;
        float v2[64];  // this thread's 64 columns of layer 2, one TMEM load
        tc::tmem_ld64(tmem + lane_base + (uint32_t)(kH + half * 64), v2);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = half * 4 + cc;
            const float *v = v2 + cc * 16;
            uint32_t pk[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = c * 16 + 2 * j;
                // H2 is rounded to bf16 (the stored activation); the output uses the same rounded values
                const __nv_bfloat162 h =
                    __floats2bfloat162_rn(fmaxf(v[2 * j] + S.b2[col], 0.f), fmaxf(v[2 * j + 1] + S.b2[col + 1], 0.f));
                acc += __bfloat162float(h.x) * S.w3[col] + __bfloat162float(h.y) * S.w3[col + 1];
                pk[j] = *reinterpret_cast<const uint32_t *>(&h);
            }
            if (H2out && r < R) {
                uint4 *g = reinterpret_cast<uint4 *>(H2out + r * kH + c * 16);
                g[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                g[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        if (half) S.ypart[row] = acc;
        tc::tc_fence_before();
        __syncthreads();  // TMEM and H1 are rewritten by the next tile; ypart is complete
        if (!half && r < R) y[r] = (acc + S.ypart[row]) + b3;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1u);
        // bounded waits for what this block still has in flight
        if (mma_pending) tc::mbar_wait(&S.bar_mma, pm, kWaitLimit);
        for (int b = 0; b < 2; ++b)
            if (x_pending[b]) tc::mbar_wait(&S.bar_x[b], px[b], kWaitLimit);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// C = A * B on the tensor cores, 128 x 128 output tiles, K in stages of 64.
// A(m, k) = A[m*sAm + k*sAk], B(k, n) = B[k*sBk + n*sBn] (bf16, any strides;
// rows beyond M or N and K beyond the block's range are zero).  The threads
// stage both operands into the K-block layout, one thread issues the four
// K = 16 MMAs of a stage into the TMEM accumulator, and the epilogue (thread t
// = output row t) either atomically adds into fp32 C (grid.z splits K: weight
// gradients) or writes bf16 C * [mask > 0] (grid.z = 1).
enum { kEpiAtomic = 0, kEpiMaskBf16 = 1 };
constexpr int kGT = 128, kGKs = 64;

struct GemmSmem {
    bf16 a[kGT * kGKs];
    bf16 b[kGT * kGKs];
    uint64_t bar;
    uint32_t tmem;
};
// at most three blocks (3 x 128 TMEM columns) per SM; descriptor reach as in FwdSmem
constexpr int kGemmSmemBytes = 64 * 1024;
static_assert(sizeof(GemmSmem) + 1024 <= kGemmSmemBytes, "gemm shared memory");
static_assert(offsetof(GemmSmem, b) + 3 * 4096 + 15 * 2048 + 256 <= kGemmSmemBytes, "descriptor reach");

// One operand row (index `row` of the tile) for K positions [k0, k0 + 64):
// element (row, k) = P[row_off + k * sk]; lanes beyond `limit` are zero.
__device__ __forceinline__ void stage_row(bf16 *tile, int row, const bf16 *P, int64_t row_off, int64_t sk, bool valid,
                                          int64_t k0, int64_t k_end)
{
    uint4 *t = reinterpret_cast<uint4 *>(tile);
    const unsigned short *q = reinterpret_cast<const unsigned short *>(P);
#pragma unroll 1
    for (int kb = 0; kb < kGKs / 8; ++kb) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t k = k0 + kb * 8 + 2 * j;
            const uint32_t lo = (valid && k < k_end) ? q[row_off + k * sk] : 0u;
            const uint32_t hi = (valid && k + 1 < k_end) ? q[row_off + (k + 1) * sk] : 0u;
            w[j] = lo | (hi << 16);
        }
        t[kb * kGT + row] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <int EPI>
__global__ void __launch_bounds__(kGT, 1)
    k_gemm(int64_t M, int64_t N, int64_t K, const bf16 *A, int64_t sAm, int64_t sAk, const bf16 *B, int64_t sBk,
           int64_t sBn, float *C, int64_t ldc, const bf16 *mask, bf16 *outb, int64_t kchunk, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char dsm[];
    GemmSmem &S = *reinterpret_cast<GemmSmem *>(dsm);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        tc::mbar_init(&S.bar, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, kGT);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const int64_t m0 = (int64_t)blockIdx.y * kGT, n0 = (int64_t)blockIdx.x * kGT;
    const int64_t k_begin = (int64_t)blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    const uint32_t id = tc::idesc_bf16(kGT, kGT);
    const int64_t gm = m0 + tid, gn = n0 + tid;
    bool ok = true, mma_pending = false, any = false;
    uint32_t pm = 0;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += kGKs) {
        stage_row(S.a, tid, A, gm * sAm, sAk, gm < M, k0, k_end);
        stage_row(S.b, tid, B, gn * sBn, sBk, gn < N, k0, k_end);
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll
            for (int k = 0; k < kGKs / 16; ++k)
                tc::mma_bf16(tmem, tc::smem_desc(S.a + k * 2 * kGT * 8, kGT * 16, 128),
                             tc::smem_desc(S.b + k * 2 * kGT * 8, kGT * 16, 128), id, (any || k > 0) ? 1u : 0u);
            tc::mma_commit(&S.bar);
        }
        any = true;
        mma_pending = true;
        ok = __syncthreads_and(tc::mbar_wait(&S.bar, pm, kWaitLimit));
        if (!ok) break;
        pm ^= 1;
        mma_pending = false;
    }
    if (ok && any) {
        tc::tc_fence_after();
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < kGT / 16; ++c) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)(c * 16), v);
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int64_t n = n0 + c * 16 + j;
                if (n >= N) continue;
                if (EPI == kEpiAtomic) {
                    atomicAdd(C + gm * ldc + n, v[j]);
                } else {
                    const bool on = __bfloat162float(mask[gm * ldc + n]) > 0.f;
                    outb[gm * ldc + n] = __float2bfloat16_rn(on ? v[j] : 0.f);
                }
            }
        }
    } else if (!ok) {
        if (tid == 0) atomicExch(err, 1u);
        if (mma_pending) tc::mbar_wait(&S.bar, pm, kWaitLimit);
    }
    if (EPI == kEpiMaskBf16 && !any && gm < M)  // empty K: the product is zero
        for (int64_t n = n0; n < min(N, n0 + kGT); ++n) outb[gm * ldc + n] = __float2bfloat16_rn(0.f);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kGT);
}

// out[j] += sum over rows of Z[r][j] (bf16 [R][128]); one warp per row, four
// columns per lane.
__global__ void k_colsum_bf16(const bf16 *Z, int64_t R, float *out)
{
    __shared__ float cs[kH];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) cs[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += __bfloat162float(Z[r * kH + lane + 32 * q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(&cs[lane + 32 * q], acc[q]);
    __syncthreads();
    for (int i = threadIdx.x; i < kH; i += blockDim.x) atomicAdd(out + i, cs[i]);
}

// dy = (y - t)/R; loss += (y - t)^2 / (2R); dZ2 = dy (x) w3 * [H2 > 0] (bf16);
// grad w3 += H2^T dy, b3 += sum dy, b2 += column sums of dZ2.
__global__ void k_mlp_out_grad(const float *y, const float *tgt, const int32_t *rows_idx, int64_t R, const bf16 *H2,
                               const float *p, bf16 *dZ2, float *grad, float *loss)
{
    __shared__ float gw3[kH], gb2[kH];
    __shared__ float gb3, ls;
    for (int i = threadIdx.x; i < kH; i += blockDim.x) gw3[i] = gb2[i] = 0.f;
    if (threadIdx.x == 0) gb3 = ls = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float accw3[4] = {0, 0, 0, 0}, accb2[4] = {0, 0, 0, 0}, accb3 = 0.f, accl = 0.f;
    for (int64_t r = w0; r < R; r += nw) {      // one warp per row, 4 columns per lane
        const int64_t src = rows_idx ? rows_idx[r] : r;
        const float diff = y[r] - tgt[src];
        const float dy = diff / (float)R;
        if (lane == 0) {
            accb3 += dy;
            accl += diff * diff / (2.f * (float)R);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            const float h = __bfloat162float(H2[r * kH + j]);
            const float d = h > 0.f ? dy * p[kOffW3 + j] : 0.f;
            const bf16 db = __float2bfloat16_rn(d);
            dZ2[r * kH + j] = db;
            accw3[q] += h * dy;
            accb2[q] += __bfloat162float(db);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        atomicAdd(&gw3[lane + 32 * q], accw3[q]);
        atomicAdd(&gb2[lane + 32 * q], accb2[q]);
    }
    if (lane == 0) {
        atomicAdd(&gb3, accb3);
        atomicAdd(&ls, accl);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        atomicAdd(grad + kOffW3 + i, gw3[i]);
        atomicAdd(grad + kOffB2 + i, gb2[i]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(grad + kOffB3, gb3);
        if (loss) atomicAdd(loss, ls);
    }
}

// gather X rows for the weight gradient of layer 1 (X^T dZ1 needs X by row index)
__global__ void k_gather_rows(const bf16 *X, const int32_t *rows_idx, int64_t R, bf16 *Xg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R * kF; i += (int64_t)gridDim.x * blockDim.x)
        Xg[i] = X[(int64_t)rows_idx[i / kF] * kF + i % kF];
}

// v = mu*v + clip(g); p -= lr*v; zero g; refresh the bf16 operand copies.
// Each gradient element is clipped to [-kClip, kClip] (non-finite -> 0) so a
// rare large batch cannot blow the weights up.
constexpr float kClip = 1.0f;

// W1c / W2c are the tensor-core B operands in the K-block layout (row = out,
// K = in); W2b = W2 row-major (B operand of dZ2 W2^T).
__global__ void k_mlp_sgd(float *p, float *v, float *gr, float lr, float mu, bf16 *W1c, bf16 *W2c, bf16 *W2b)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNumParams; i += gridDim.x * blockDim.x) {
        if (lr != 0.f || mu != 0.f) {
            float gi = gr[i];
            gi = isfinite(gi) ? fminf(fmaxf(gi, -kClip), kClip) : 0.f;
            v[i] = mu * v[i] + gi;
            p[i] -= lr * v[i];
        }
        gr[i] = 0.f;
        const float w = p[i];
        if (i < kOffB1) {                         // W1[in][out]
            const int in = i / kH, out = i % kH;
            W1c[kblk(out, in, kH)] = __float2bfloat16_rn(w);
        } else if (i >= kOffW2 && i < kOffB2) {   // W2[in][out]
            const int j = i - kOffW2, in = j / kH, out = j % kH;
            W2c[kblk(out, in, kH)] = __float2bfloat16_rn(w);
            W2b[j] = __float2bfloat16_rn(w);
        }
    }
}

// keys for the top-k: order-preserving map of float scores to unsigned
__global__ void k_score_keys(const float *sc, int32_t n, unsigned long long *keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = __float_as_uint(sc[i]);
        b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        keys[i] = (unsigned long long)b;
    }
}

// Spread selection: keys hold (order-preserving score << 32) | (~id); a
// vertex already taken or excluded has key 0.  One pass finds the largest
// key (the highest score, ties by smaller id); one block then takes that
// vertex and excludes its in- and out-neighbours.
__global__ void k_spread_keys(const float *sc, int32_t n, unsigned long long *keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = __float_as_uint(sc[i]);
        b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        const float f = sc[i];
        keys[i] = (f != f || b == 0x007FFFFFu) ? 0ull  // NaN or -inf: never taken
                                               : ((unsigned long long)b << 32) | (uint32_t)~(uint32_t)i;
    }
}

__global__ void k_spread_max(const unsigned long long *keys, int32_t n, unsigned long long *best)
{
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = keys[i] > m ? keys[i] : m;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(best, m);
}

__global__ void k_spread_take(DevGraph g, unsigned long long *keys, unsigned long long *best, int32_t *out, int32_t i,
                              int spread)
{
    const unsigned long long b = *best;
    __syncthreads();
    if (threadIdx.x == 0) *best = 0;
    if (!b) {
        if (threadIdx.x == 0) out[i] = -1;  // fewer candidates than slots
        return;
    }
    const int32_t x = (int32_t)~(uint32_t)(b & 0xffffffffull);
    if (threadIdx.x == 0) {
        out[i] = x;
        keys[x] = 0;
    }
    if (!spread) return;
    for (int dir = 0; dir < 2; ++dir) {
        const AdjRange r = adj_of(g, dir, x);
        for (int32_t e = threadIdx.x; e < r.bd + r.od; e += blockDim.x) keys[adj_at(g, dir, r, e)] = 0;
    }
}

// A vertex in the strongly connected component of one of the index's first
// `slots` landmarks (its DL_in and DL_out share that landmark's bit) is never
// taken: every pair it connects, the landmark connects too.
__global__ void k_drop_covered(const uint64_t *rec, int32_t hs, int32_t wd, int32_t slots, int32_t n,
                               unsigned long long *keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *p = rec + (size_t)i * 2 * hs;
        bool cov = false;
        for (int w = 0; w < wd && w * 64 < slots; ++w) {
            const int rem = slots - w * 64;
            const uint64_t mask = rem >= 64 ? ~0ull : ((1ull << rem) - 1);
            cov |= (p[w] & p[hs + w] & mask) != 0;
        }
        if (cov) keys[i] = 0;
    }
}

static unsigned grid_cap(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace dbl

// ------------------------------------------------------------ the network object
struct dbl_mlp {
    float *p = nullptr, *v = nullptr, *gr = nullptr;  // fp32 parameters, momentum, gradients
    dbl::bf16 *W1c = nullptr, *W2c = nullptr, *W2b = nullptr;
    dbl::bf16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *Xg = nullptr;
    float *y = nullptr;
    uint32_t *d_err = nullptr;  // raised by a tensor-core kernel whose bounded wait ran out
    int64_t cap_rows = 0;
    std::string err;
};

using namespace dbl;

static dbl_status mlp_fail(dbl_mlp *m, dbl_status st, const std::string &msg)
{
    if (m) m->err = msg;
    return st;
}

static dbl_status mlp_alloc(dbl_mlp *m, void **p, size_t bytes, cudaStream_t s)
{
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e) {
        cudaGetLastError();
        return mlp_fail(m, DBL_ERR_OOM, std::string("mlp allocation: ") + cudaGetErrorString(e));
    }
    return DBL_OK;
}

static dbl_status mlp_scratch(dbl_mlp *m, int64_t rows, cudaStream_t s)
{
    if (rows <= m->cap_rows) return DBL_OK;
    void *old[6] = {m->H1, m->H2, m->dZ2, m->dZ1, m->Xg, m->y};
    for (void *p : old)
        if (p) cudaFreeAsync(p, s);
    dbl_status st;
    if ((st = mlp_alloc(m, (void **)&m->H1, sizeof(bf16) * rows * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->H2, sizeof(bf16) * rows * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->dZ2, sizeof(bf16) * rows * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->dZ1, sizeof(bf16) * rows * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->Xg, sizeof(bf16) * rows * kF, s)) ||
        (st = mlp_alloc(m, (void **)&m->y, sizeof(float) * rows, s)))
        return st;
    m->cap_rows = rows;
    return DBL_OK;
}

static MlpDev mlp_dev(const dbl_mlp *m) { return MlpDev{m->W1c, m->W2c, m->p}; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        cudaGetLastError();
    }
    return fn;
}

// X [R][16] bf16 as a 3-D tensor (k % 8, row, k / 8) with byte strides
// (32, 16): a box of (8, 128, 2) lands in shared memory as [2][128][8], the
// K-block layout of a 128 x 16 operand tile.  Rows beyond R read as zero.
static bool x_tensor_map(const bf16 *X, int64_t R, CUtensorMap *map)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[3] = {8, (cuuint64_t)R, 2};
    const cuuint64_t strides[2] = {kF * sizeof(bf16), 8 * sizeof(bf16)};
    const cuuint32_t box[3] = {8, kTileR, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)X, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool set_smem_attrs()
{
    static int done = 0;
    if (!done) {
        bool ok = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmemBytes) ==
                      cudaSuccess &&
                  cudaFuncSetAttribute(k_gemm<kEpiAtomic>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kGemmSmemBytes) == cudaSuccess &&
                  cudaFuncSetAttribute(k_gemm<kEpiMaskBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kGemmSmemBytes) == cudaSuccess;
        done = ok ? 1 : -1;
    }
    return done == 1;
}

// Contiguous rows whose base is 16-byte aligned go through the tensor copy;
// gathered (rows_idx) or unaligned rows are staged by the threads.
static dbl_status launch_forward(dbl_mlp *m, const bf16 *X, const int32_t *idx, int64_t R, float *y, bf16 *H1,
                                 bf16 *H2, cudaStream_t s)
{
    if (!set_smem_attrs()) return mlp_fail(m, DBL_ERR_CUDA, "mlp: shared-memory attribute refused");
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    int use_tma = 0;
    if (!idx && ((uintptr_t)X & 15u) == 0) {
        if (!x_tensor_map(X, R, &map)) return mlp_fail(m, DBL_ERR_CUDA, "mlp: cuTensorMapEncodeTiled failed");
        use_tma = 1;
    }
    const int64_t tiles = (R + kTileR - 1) / kTileR;
    int64_t blocks = (int64_t)num_sms() * 2;
    if (blocks > tiles) blocks = tiles;
    k_mlp_forward<<<(unsigned)(blocks < 1 ? 1 : blocks), kFwdThreads, kFwdSmemBytes, s>>>(map, use_tma, mlp_dev(m), X, idx,
                                                                                     R, y, H1, H2, m->d_err);
    return DBL_OK;
}

template <int EPI>
static void launch_gemm(dbl_mlp *m, int64_t M, int64_t N, int64_t K, const bf16 *A, int64_t sAm, int64_t sAk,
                        const bf16 *B, int64_t sBk, int64_t sBn, float *C, int64_t ldc, const bf16 *mask, bf16 *outb,
                        int64_t kchunk, cudaStream_t s)
{
    const dim3 grid((unsigned)((N + kGT - 1) / kGT), (unsigned)((M + kGT - 1) / kGT),
                    (unsigned)((K + kchunk - 1) / kchunk));
    k_gemm<EPI><<<grid, kGT, kGemmSmemBytes, s>>>(M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, mask, outb, kchunk,
                                                   m->d_err);
}

// Gradients of the mean squared error / 2 over R rows into m->gr (zeroed by the previous SGD call).
static dbl_status mlp_backward(dbl_mlp *m, const bf16 *X, const float *tgt, const int32_t *idx, int64_t R,
                               float *loss, cudaStream_t s)
{
    dbl_status st = mlp_scratch(m, R, s);
    if (st) return st;
    if ((st = launch_forward(m, X, idx, R, m->y, m->H1, m->H2, s))) return st;
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), s);
    k_mlp_out_grad<<<grid_cap(R * 32, 256), 256, 0, s>>>(m->y, tgt, idx, R, m->H2, m->p, m->dZ2, m->gr, loss);
    const int64_t kchunk = 1024;
    // dW2 = H1^T dZ2: M = 128 (in), N = 128 (out), K = R
    launch_gemm<kEpiAtomic>(m, kH, kH, R, m->H1, 1, kH, m->dZ2, kH, 1, m->gr + kOffW2, kH, nullptr, nullptr, kchunk,
                            s);
    // dZ1 = (dZ2 W2^T) * [H1 > 0]: M = R, N = 128 (in), K = 128 (out); B(k=out, n=in) = W2[in][out]
    launch_gemm<kEpiMaskBf16>(m, R, kH, kH, m->dZ2, kH, 1, m->W2b, 1, kH, nullptr, kH, m->H1, m->dZ1, kH, s);
    // db1 = column sums of dZ1
    k_colsum_bf16<<<grid_cap(R * 32, 256), 256, 0, s>>>(m->dZ1, R, m->gr + kOffB1);
    // dW1 = X^T dZ1: M = 16, N = 128, K = R
    const bf16 *Xr = X;
    if (idx) {
        k_gather_rows<<<grid_cap(R * kF, 256), 256, 0, s>>>(X, idx, R, m->Xg);
        Xr = m->Xg;
    }
    launch_gemm<kEpiAtomic>(m, kF, kH, R, Xr, 1, kF, m->dZ1, kH, 1, m->gr + kOffW1, kH, nullptr, nullptr, kchunk, s);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, std::string("mlp backward: ") + cudaGetErrorString(e)) : DBL_OK;
}

extern "C" {

dbl_status dbl_features(dbl_index *ix, uint16_t *feat, void *stream)
{
    if (!ix || !feat) return dbl::fail(ix, DBL_ERR_INVALID, "features: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (dbl_status fs = flush_insertions(ix, s)) return fs;  // queued batches (DBL_FLAG_DEFER) first
    dbl_status st = dbl::features(ix, (bf16 *)feat, s);
    if (st) return st;
    return (ix->opt.flags & DBL_FLAG_ASYNC) ? DBL_OK : read_status(ix, s);
}

dbl_status dbl_coverage(dbl_index *ix, const int32_t *u, const int32_t *v, const uint8_t *reach, int64_t pairs,
                        int32_t base_slots, uint32_t *count, float *target, int64_t *kept, void *stream)
{
    if (!ix || !count || pairs < 0 || (pairs > 0 && (!u || !v)) || base_slots < 0 || base_slots > ix->k)
        return dbl::fail(ix, DBL_ERR_INVALID, "coverage: bad arguments");
    if (ix->poisoned) return dbl::fail(ix, DBL_ERR_POISONED, "index poisoned");
    cudaStream_t s = (cudaStream_t)stream;
    if (dbl_status fs = flush_insertions(ix, s)) return fs;  // queued batches (DBL_FLAG_DEFER) first
    dbl_status st = dbl::coverage(ix, u, v, reach, pairs, base_slots, count, kept, s);
    if (st) return st;
    if (target) {
        k_cov_targets<<<1, 1024, 0, s>>>(count, ix->n, target);
        ++ix->launches;
    }
    return read_status(ix, s);
}

// Greedy selection over the score keys: k times the largest remaining key,
// then (spread) its neighbours excluded.
static dbl_status select_greedy(dbl_index *ix, const float *scores, int32_t k, int32_t covered_slots, int spread,
                                int32_t *out, cudaStream_t s)
{
    unsigned long long *keys = nullptr;
    dbl_status st = alloc_buf(ix, (void **)&keys, sizeof(unsigned long long) * ((size_t)ix->n + 1), s);
    if (st) return st;
    unsigned long long *best = keys + ix->n;
    cudaMemsetAsync(best, 0, sizeof(unsigned long long), s);
    k_spread_keys<<<grid_cap(ix->n, kBlock), kBlock, 0, s>>>(scores, ix->n, keys);
    ++ix->launches;
    if (covered_slots > 0) {
        k_drop_covered<<<grid_cap(ix->n, kBlock), kBlock, 0, s>>>(ix->rec, ix->hs, ix->wd,
                                                                  std::min<int32_t>(covered_slots, ix->k), ix->n, keys);
        ++ix->launches;
    }
    const DevGraph g = dev_graph(ix);
    for (int32_t i = 0; i < k; ++i) {
        k_spread_max<<<grid_cap(ix->n, kBlock), kBlock, 0, s>>>(keys, ix->n, best);
        k_spread_take<<<1, kBlock, 0, s>>>(g, keys, best, out, i, spread);
        ix->launches += 2;
    }
    free_buf(ix, keys, s);
    cudaError_t e = cudaGetLastError();
    if (e) return cuda_fail(ix, e, "select");
    return read_status(ix, s);
}

dbl_status dbl_select_spread(dbl_index *ix, const float *scores, int32_t k, int32_t *out, void *stream)
{
    if (!ix || !scores || !out || k <= 0) return dbl::fail(ix, DBL_ERR_INVALID, "select_spread: bad arguments");
    return select_greedy(ix, scores, k, 0, 1, out, (cudaStream_t)stream);
}

dbl_status dbl_select_uncovered(dbl_index *ix, const float *scores, int32_t k, int32_t covered_slots, int32_t spread,
                                int32_t *out, void *stream)
{
    if (!ix || !scores || !out || k <= 0 || covered_slots < 0)
        return dbl::fail(ix, DBL_ERR_INVALID, "select_uncovered: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (dbl_status fs = flush_insertions(ix, s)) return fs;  // the labels it reads include queued batches
    return select_greedy(ix, scores, k, covered_slots, spread ? 1 : 0, out, s);
}

dbl_status dbl_select_by_score(dbl_index *ix, const float *scores, int32_t k, int32_t *out, void *stream)
{
    if (!ix || !scores || !out || k <= 0) return dbl::fail(ix, DBL_ERR_INVALID, "select_by_score: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *keys = nullptr;
    dbl_status st = alloc_buf(ix, (void **)&keys, sizeof(unsigned long long) * (size_t)ix->n + 16, s);
    if (st) return st;
    k_score_keys<<<grid_cap(ix->n, kBlock), kBlock, 0, s>>>(scores, ix->n, keys);
    ++ix->launches;
    st = select_top(ix, nullptr, nullptr, keys, ix->n, k, out, s);
    free_buf(ix, keys, s);
    if (st) return st;
    return read_status(ix, s);
}

dbl_status dbl_mlp_create(const float *params_host, dbl_mlp **out, void *stream)
{
    if (!out || !params_host) return DBL_ERR_INVALID;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    dbl_mlp *m = new dbl_mlp();
    dbl_status st;
    if ((st = mlp_alloc(m, (void **)&m->p, sizeof(float) * kNumParams, s)) ||
        (st = mlp_alloc(m, (void **)&m->v, sizeof(float) * kNumParams, s)) ||
        (st = mlp_alloc(m, (void **)&m->gr, sizeof(float) * kNumParams, s)) ||
        (st = mlp_alloc(m, (void **)&m->W1c, sizeof(bf16) * kF * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->W2c, sizeof(bf16) * kH * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->d_err, 16, s)) ||
        (st = mlp_alloc(m, (void **)&m->W2b, sizeof(bf16) * kH * kH, s))) {
        dbl_mlp_destroy(m, stream);
        return st;
    }
    cudaMemcpyAsync(m->p, params_host, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(m->v, 0, sizeof(float) * kNumParams, s);
    cudaMemsetAsync(m->gr, 0, sizeof(float) * kNumParams, s);
    cudaMemsetAsync(m->d_err, 0, 16, s);
    k_mlp_sgd<<<(kNumParams + 255) / 256, 256, 0, s>>>(m->p, m->v, m->gr, 0.f, 0.f, m->W1c, m->W2c, m->W2b);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) {
        dbl_mlp_destroy(m, stream);
        return DBL_ERR_CUDA;
    }
    *out = m;
    return DBL_OK;
}

void dbl_mlp_destroy(dbl_mlp *m, void *stream)
{
    if (!m) return;
    cudaStream_t s = (cudaStream_t)stream;
    void *ps[] = {m->p, m->v, m->gr, m->W1c, m->W2c, m->W2b, m->H1, m->H2, m->dZ2, m->dZ1, m->Xg, m->y, m->d_err};
    for (void *p : ps)
        if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
    delete m;
}

dbl_status dbl_mlp_params(dbl_mlp *m, float *params_host, void *stream)
{
    if (!m || !params_host) return DBL_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyAsync(params_host, m->p, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, s);
    return dbl_mlp_sync(m, stream);
}

dbl_status dbl_mlp_forward(dbl_mlp *m, const uint16_t *X, const int32_t *rows_idx, int64_t rows, float *y, void *stream)
{
    if (!m || !X || !y || rows < 0) return mlp_fail(m, DBL_ERR_INVALID, "mlp_forward: bad arguments");
    if ((uintptr_t)X & 15u) return mlp_fail(m, DBL_ERR_INVALID, "mlp: X must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (rows) {
        dbl_status st = launch_forward(m, (const bf16 *)X, rows_idx, rows, y, nullptr, nullptr, s);
        if (st) return st;
    }
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e)) : DBL_OK;
}

dbl_status dbl_mlp_gradients(dbl_mlp *m, const uint16_t *X, const float *target, const int32_t *rows_idx, int64_t rows,
                             float *grads, float *loss, void *stream)
{
    if (!m || !X || !target || !grads || rows <= 0) return mlp_fail(m, DBL_ERR_INVALID, "mlp_gradients: bad arguments");
    if ((uintptr_t)X & 15u) return mlp_fail(m, DBL_ERR_INVALID, "mlp: X must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    dbl_status st = mlp_backward(m, (const bf16 *)X, target, rows_idx, rows, loss, s);
    if (st) return st;
    cudaMemcpyAsync(grads, m->gr, sizeof(float) * kNumParams, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(m->gr, 0, sizeof(float) * kNumParams, s);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e)) : DBL_OK;
}

dbl_status dbl_mlp_train_step(dbl_mlp *m, const uint16_t *X, const float *target, const int32_t *rows_idx, int64_t rows,
                              float lr, float momentum, float *loss, void *stream)
{
    if (!m || !X || !target || rows <= 0) return mlp_fail(m, DBL_ERR_INVALID, "mlp_train_step: bad arguments");
    if ((uintptr_t)X & 15u) return mlp_fail(m, DBL_ERR_INVALID, "mlp: X must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    dbl_status st = mlp_backward(m, (const bf16 *)X, target, rows_idx, rows, loss, s);
    if (st) return st;
    k_mlp_sgd<<<(kNumParams + 255) / 256, 256, 0, s>>>(m->p, m->v, m->gr, lr, momentum, m->W1c, m->W2c, m->W2b);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e)) : DBL_OK;
}

dbl_status dbl_mlp_sync(dbl_mlp *m, void *stream)
{
    if (!m) return DBL_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t flag = 0;
    cudaMemcpyAsync(&flag, m->d_err, sizeof(flag), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e));
    if (flag) return mlp_fail(m, DBL_ERR_TIMEOUT, "mlp: a tensor-core wait ran out; outputs are invalid");
    return DBL_OK;
}

const char *dbl_mlp_last_error(const dbl_mlp *m) { return m ? m->err.c_str() : ""; }

}  // extern "C"
