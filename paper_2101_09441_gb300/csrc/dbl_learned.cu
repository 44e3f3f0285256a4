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
//   MLP        bf16 operands, fp32 accumulate, mma.sync m16n8k16 tensor-core
//              tiles; a fused forward (both hidden layers stay in registers)
//              and a backward of three GEMMs with split-K reductions
//   selection  top-k by score with the landmark radix select
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dbl_frontier.cuh"
#include "dbl_internal.cuh"
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
__global__ void k_features(DevGraph g, const uint64_t *rec, int32_t hs, int32_t wd, int32_t wb, const uint8_t *mark,
                           bf16 *out)
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
            for (int w = 0; w < wd; ++w) {
                pc[0] += __popcll(p[w]);
                pc[1] += __popcll(p[hs + w]);
            }
            for (int w = 0; w < wb; ++w) {
                pc[2] += __popcll(p[wd + w]);
                pc[3] += __popcll(p[hs + wd + w]);
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
    k_features<<<(unsigned)blocks, kBlock, 0, s>>>(dev_graph(ix), ix->rec, ix->hs, ix->wd, ix->wb, mark, out);
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

// ------------------------------------------------------------ tensor-core tiles
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// D = A(16x16, row) * B(16x8, col) + C, bf16 inputs, fp32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kH = 128;       // hidden width
constexpr int kF = 16;        // features
constexpr int kW1Pitch = kF + 8;    // smem pitch (bf16) of W1t rows: [out][in]
constexpr int kW2Pitch = kH + 8;    // smem pitch (bf16) of W2t rows: [out][in]

// Parameter offsets in the flat fp32 vector (18,817 values).
constexpr int kOffW1 = 0;                     // [16][128]  (in x out)
constexpr int kOffB1 = kOffW1 + kF * kH;      // [128]
constexpr int kOffW2 = kOffB1 + kH;           // [128][128] (in x out)
constexpr int kOffB2 = kOffW2 + kH * kH;      // [128]
constexpr int kOffW3 = kOffB2 + kH;           // [128]
constexpr int kOffB3 = kOffW3 + kH;           // [1]
constexpr int kNumParams = kOffB3 + 1;

struct MlpDev {
    const bf16 *W1t;      // [128][16]  out-major (B operand of layer 1)
    const bf16 *W2t;      // [128][128] out-major (B operand of layer 2)
    const float *p;       // fp32 parameters (biases, w3, b3)
};

// Fused forward: each warp takes 16 rows; both hidden layers stay in
// registers (the accumulator fragment of two n8 tiles is exactly the A
// fragment of the next k16 step).  Optionally stores H1, H2 (bf16) for the
// backward pass.  rows_idx (optional) gathers the input rows.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpDev m, const bf16 *X, const int32_t *rows_idx, int64_t R,
                                                     float *y, bf16 *H1out, bf16 *H2out)
{
    __shared__ __align__(16) bf16 w1s[kH * kW1Pitch];
    __shared__ __align__(16) bf16 w2s[kH * kW2Pitch];
    __shared__ float b1s[kH], b2s[kH], w3s[kH];
    for (int i = threadIdx.x; i < kH * kF; i += blockDim.x) w1s[(i / kF) * kW1Pitch + i % kF] = m.W1t[i];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) w2s[(i / kH) * kW2Pitch + i % kH] = m.W2t[i];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        b1s[i] = m.p[kOffB1 + i];
        b2s[i] = m.p[kOffB2 + i];
        w3s[i] = m.p[kOffW3 + i];
    }
    const float b3 = m.p[kOffB3];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 16; r0 < R; r0 += nwarp * 16) {
        const int64_t ra = r0 + g, rb = r0 + g + 8;
        const int64_t xa = ra < R ? (rows_idx ? rows_idx[ra] : ra) : -1;
        const int64_t xb = rb < R ? (rows_idx ? rows_idx[rb] : rb) : -1;
        uint32_t a[4];
        const uint32_t *Xa = reinterpret_cast<const uint32_t *>(X + (xa >= 0 ? xa : 0) * kF);
        const uint32_t *Xb = reinterpret_cast<const uint32_t *>(X + (xb >= 0 ? xb : 0) * kF);
        a[0] = xa >= 0 ? Xa[t] : 0u;        // row g,   cols 2t..2t+1
        a[1] = xb >= 0 ? Xb[t] : 0u;        // row g+8, cols 2t..2t+1
        a[2] = xa >= 0 ? Xa[t + 4] : 0u;    // row g,   cols 2t+8..
        a[3] = xb >= 0 ? Xb[t + 4] : 0u;    // row g+8, cols 2t+8..
        // layer 1 -> H1 as layer-2 A fragments
        uint32_t h1[8][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const bf16 *wb = w1s + (nt * 8 + g) * kW1Pitch;
            mma_bf16(c, a, *reinterpret_cast<const uint32_t *>(wb + 2 * t),
                     *reinterpret_cast<const uint32_t *>(wb + 2 * t + 8));
            const int col = nt * 8 + 2 * t;
            const float z0 = fmaxf(c[0] + b1s[col], 0.f), z1 = fmaxf(c[1] + b1s[col + 1], 0.f);
            const float z2 = fmaxf(c[2] + b1s[col], 0.f), z3 = fmaxf(c[3] + b1s[col + 1], 0.f);
            const int kt = nt >> 1;
            if ((nt & 1) == 0) {
                h1[kt][0] = pack_bf16(z0, z1);
                h1[kt][1] = pack_bf16(z2, z3);
            } else {
                h1[kt][2] = pack_bf16(z0, z1);
                h1[kt][3] = pack_bf16(z2, z3);
            }
        }
        if (H1out) {
#pragma unroll
            for (int kt = 0; kt < 8; ++kt) {
                const int col = kt * 16 + 2 * t;
                if (ra < R) {
                    *reinterpret_cast<uint32_t *>(H1out + ra * kH + col) = h1[kt][0];
                    *reinterpret_cast<uint32_t *>(H1out + ra * kH + col + 8) = h1[kt][2];
                }
                if (rb < R) {
                    *reinterpret_cast<uint32_t *>(H1out + rb * kH + col) = h1[kt][1];
                    *reinterpret_cast<uint32_t *>(H1out + rb * kH + col + 8) = h1[kt][3];
                }
            }
        }
        // layer 2 and the output dot product
        float ya = 0.f, yb = 0.f;
#pragma unroll 4
        for (int nt = 0; nt < 16; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const bf16 *wb = w2s + (nt * 8 + g) * kW2Pitch;
#pragma unroll
            for (int kt = 0; kt < 8; ++kt)
                mma_bf16(c, h1[kt], *reinterpret_cast<const uint32_t *>(wb + kt * 16 + 2 * t),
                         *reinterpret_cast<const uint32_t *>(wb + kt * 16 + 2 * t + 8));
            const int col = nt * 8 + 2 * t;
            // H2 is rounded to bf16 (the stored activation); the output uses the same rounded values
            const __nv_bfloat162 ha = __floats2bfloat162_rn(fmaxf(c[0] + b2s[col], 0.f), fmaxf(c[1] + b2s[col + 1], 0.f));
            const __nv_bfloat162 hb = __floats2bfloat162_rn(fmaxf(c[2] + b2s[col], 0.f), fmaxf(c[3] + b2s[col + 1], 0.f));
            ya += __bfloat162float(ha.x) * w3s[col] + __bfloat162float(ha.y) * w3s[col + 1];
            yb += __bfloat162float(hb.x) * w3s[col] + __bfloat162float(hb.y) * w3s[col + 1];
            if (H2out) {
                if (ra < R) *reinterpret_cast<__nv_bfloat162 *>(H2out + ra * kH + col) = ha;
                if (rb < R) *reinterpret_cast<__nv_bfloat162 *>(H2out + rb * kH + col) = hb;
            }
        }
        ya += __shfl_xor_sync(kFull, ya, 1);
        ya += __shfl_xor_sync(kFull, ya, 2);
        yb += __shfl_xor_sync(kFull, yb, 1);
        yb += __shfl_xor_sync(kFull, yb, 2);
        if (t == 0) {
            if (ra < R) y[ra] = ya + b3;
            if (rb < R) y[rb] = yb + b3;
        }
    }
}

// Generic C = A * B on tensor cores, 64x64 tiles, BK = 32, 4 warps (32x32 each).
// A(m, k) = A[m*sAm + k*sAk], B(k, n) = B[k*sBk + n*sBn] (bf16, any strides).
// grid.z splits K; the epilogue either atomically adds into fp32 C (split-K
// reductions of weight gradients) or writes bf16 C * [mask > 0] and adds the
// column sums of that product into colsum (fp32).
enum { kEpiAtomic = 0, kEpiMaskBf16 = 1 };
constexpr int kGM = 64, kGN = 64, kGK = 32, kGPitch = kGK + 8;

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(int64_t M, int64_t N, int64_t K, const bf16 *A, int64_t sAm, int64_t sAk,
                                              const bf16 *B, int64_t sBk, int64_t sBn, float *C, int64_t ldc,
                                              const bf16 *mask, bf16 *outb, float *colsum, int64_t kchunk)
{
    __shared__ __align__(16) bf16 As[kGM * kGPitch];
    __shared__ __align__(16) bf16 Bs[kGN * kGPitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int64_t m0 = (int64_t)blockIdx.y * kGM, n0 = (int64_t)blockIdx.x * kGN;
    const int64_t k_begin = (int64_t)blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (int64_t k0 = k_begin; k0 < k_end; k0 += kGK) {
        for (int i = threadIdx.x; i < kGM * kGK; i += blockDim.x) {
            const int r = i / kGK, c = i % kGK;
            const int64_t gm = m0 + r, gk = k0 + c;
            As[r * kGPitch + c] = (gm < M && gk < k_end) ? A[gm * sAm + gk * sAk] : zero;
            const int64_t gn = n0 + r;
            Bs[r * kGPitch + c] = (gn < N && gk < k_end) ? B[gk * sBk + gn * sBn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; kk += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const bf16 *p = As + (wm + mt * 16 + g) * kGPitch + kk + 2 * t;
                a[mt][0] = *reinterpret_cast<const uint32_t *>(p);
                a[mt][1] = *reinterpret_cast<const uint32_t *>(p + 8 * kGPitch);
                a[mt][2] = *reinterpret_cast<const uint32_t *>(p + 8);
                a[mt][3] = *reinterpret_cast<const uint32_t *>(p + 8 * kGPitch + 8);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const bf16 *p = Bs + (wn + nt * 8 + g) * kGPitch + kk + 2 * t;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(p);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(p + 8);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b0, b1);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        float cs[2] = {0.f, 0.f};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t gm = m0 + wm + mt * 16 + g + (q >= 2 ? 8 : 0);
                const int64_t gn = n0 + wn + nt * 8 + 2 * t + (q & 1);
                if (gm >= M || gn >= N) continue;
                if (EPI == kEpiAtomic) {
                    atomicAdd(C + gm * ldc + gn, acc[mt][nt][q]);
                } else {
                    const bool on = __bfloat162float(mask[gm * ldc + gn]) > 0.f;
                    const bf16 v = __float2bfloat16_rn(on ? acc[mt][nt][q] : 0.f);
                    outb[gm * ldc + gn] = v;
                    cs[q & 1] += __bfloat162float(v);
                }
            }
        }
        if (EPI == kEpiMaskBf16) {
            // reduce over the 8 row-groups g of the warp, then one atomic per column
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                cs[0] += __shfl_xor_sync(kFull, cs[0], o);
                cs[1] += __shfl_xor_sync(kFull, cs[1], o);
            }
            if (g == 0) {
                const int64_t gn = n0 + wn + nt * 8 + 2 * t;
                if (gn < N) atomicAdd(colsum + gn, cs[0]);
                if (gn + 1 < N) atomicAdd(colsum + gn + 1, cs[1]);
            }
        }
    }
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

__global__ void k_mlp_sgd(float *p, float *v, float *gr, float lr, float mu, bf16 *W1t, bf16 *W2t, bf16 *W2b)
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
        if (i < kOffB1) {                         // W1[in][out] -> W1t[out][in]
            const int in = i / kH, out = i % kH;
            W1t[out * kF + in] = __float2bfloat16_rn(w);
        } else if (i >= kOffW2 && i < kOffB2) {   // W2[in][out] -> W2t[out][in] and W2b = W2
            const int j = i - kOffW2, in = j / kH, out = j % kH;
            W2t[out * kH + in] = __float2bfloat16_rn(w);
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
    dbl::bf16 *W1t = nullptr, *W2t = nullptr, *W2b = nullptr;
    dbl::bf16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *Xg = nullptr;
    float *y = nullptr;
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

static MlpDev mlp_dev(const dbl_mlp *m) { return MlpDev{m->W1t, m->W2t, m->p}; }

static void launch_forward(dbl_mlp *m, const bf16 *X, const int32_t *idx, int64_t R, float *y, bf16 *H1, bf16 *H2,
                           cudaStream_t s)
{
    int64_t warps = (R + 15) / 16;
    int64_t blocks = (warps + 3) / 4;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_mlp_forward<<<(unsigned)(blocks < 1 ? 1 : blocks), 128, 0, s>>>(mlp_dev(m), X, idx, R, y, H1, H2);
}

// Gradients of the mean squared error / 2 over R rows into m->gr (zeroed by the previous SGD call).
static dbl_status mlp_backward(dbl_mlp *m, const bf16 *X, const float *tgt, const int32_t *idx, int64_t R,
                               float *loss, cudaStream_t s)
{
    dbl_status st = mlp_scratch(m, R, s);
    if (st) return st;
    launch_forward(m, X, idx, R, m->y, m->H1, m->H2, s);
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), s);
    k_mlp_out_grad<<<grid_cap(R * 32, 256), 256, 0, s>>>(m->y, tgt, idx, R, m->H2, m->p, m->dZ2, m->gr, loss);
    const int64_t kchunk = 1024;
    const unsigned zs = (unsigned)((R + kchunk - 1) / kchunk);
    // dW2 = H1^T dZ2: M = 128 (in), N = 128 (out), K = R
    k_gemm<kEpiAtomic><<<dim3(2, 2, zs), 128, 0, s>>>(kH, kH, R, m->H1, 1, kH, m->dZ2, kH, 1, m->gr + kOffW2, kH,
                                                      nullptr, nullptr, nullptr, kchunk);
    // dZ1 = (dZ2 W2^T) * [H1 > 0]: M = R, N = 128 (in), K = 128 (out); B(k=out, n=in) = W2[in][out]
    k_gemm<kEpiMaskBf16><<<dim3(2, (unsigned)((R + kGM - 1) / kGM), 1), 128, 0, s>>>(
        R, kH, kH, m->dZ2, kH, 1, m->W2b, 1, kH, nullptr, kH, m->H1, m->dZ1, m->gr + kOffB1, kH);
    // dW1 = X^T dZ1: M = 16, N = 128, K = R
    const bf16 *Xr = X;
    if (idx) {
        k_gather_rows<<<grid_cap(R * kF, 256), 256, 0, s>>>(X, idx, R, m->Xg);
        Xr = m->Xg;
    }
    k_gemm<kEpiAtomic><<<dim3(2, 1, zs), 128, 0, s>>>(kF, kH, R, Xr, 1, kF, m->dZ1, kH, 1, m->gr + kOffW1, kH,
                                                      nullptr, nullptr, nullptr, kchunk);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, std::string("mlp backward: ") + cudaGetErrorString(e)) : DBL_OK;
}

extern "C" {

dbl_status dbl_features(dbl_index *ix, uint16_t *feat, void *stream)
{
    if (!ix || !feat) return dbl::fail(ix, DBL_ERR_INVALID, "features: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
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
    dbl_status st = dbl::coverage(ix, u, v, reach, pairs, base_slots, count, kept, s);
    if (st) return st;
    if (target) {
        k_cov_targets<<<1, 1024, 0, s>>>(count, ix->n, target);
        ++ix->launches;
    }
    return read_status(ix, s);
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
        (st = mlp_alloc(m, (void **)&m->W1t, sizeof(bf16) * kF * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->W2t, sizeof(bf16) * kH * kH, s)) ||
        (st = mlp_alloc(m, (void **)&m->W2b, sizeof(bf16) * kH * kH, s))) {
        dbl_mlp_destroy(m, stream);
        return st;
    }
    cudaMemcpyAsync(m->p, params_host, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(m->v, 0, sizeof(float) * kNumParams, s);
    cudaMemsetAsync(m->gr, 0, sizeof(float) * kNumParams, s);
    k_mlp_sgd<<<(kNumParams + 255) / 256, 256, 0, s>>>(m->p, m->v, m->gr, 0.f, 0.f, m->W1t, m->W2t, m->W2b);
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
    void *ps[] = {m->p, m->v, m->gr, m->W1t, m->W2t, m->W2b, m->H1, m->H2, m->dZ2, m->dZ1, m->Xg, m->y};
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
    return cudaStreamSynchronize(s) ? DBL_ERR_CUDA : DBL_OK;
}

dbl_status dbl_mlp_forward(dbl_mlp *m, const uint16_t *X, const int32_t *rows_idx, int64_t rows, float *y, void *stream)
{
    if (!m || !X || !y || rows < 0) return mlp_fail(m, DBL_ERR_INVALID, "mlp_forward: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (rows) launch_forward(m, (const bf16 *)X, rows_idx, rows, y, nullptr, nullptr, s);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e)) : DBL_OK;
}

dbl_status dbl_mlp_gradients(dbl_mlp *m, const uint16_t *X, const float *target, const int32_t *rows_idx, int64_t rows,
                             float *grads, float *loss, void *stream)
{
    if (!m || !X || !target || !grads || rows <= 0) return mlp_fail(m, DBL_ERR_INVALID, "mlp_gradients: bad arguments");
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
    cudaStream_t s = (cudaStream_t)stream;
    dbl_status st = mlp_backward(m, (const bf16 *)X, target, rows_idx, rows, loss, s);
    if (st) return st;
    k_mlp_sgd<<<(kNumParams + 255) / 256, 256, 0, s>>>(m->p, m->v, m->gr, lr, momentum, m->W1t, m->W2t, m->W2b);
    cudaError_t e = cudaGetLastError();
    return e ? mlp_fail(m, DBL_ERR_CUDA, cudaGetErrorString(e)) : DBL_OK;
}

const char *dbl_mlp_last_error(const dbl_mlp *m) { return m ? m->err.c_str() : ""; }

}  // extern "C"
