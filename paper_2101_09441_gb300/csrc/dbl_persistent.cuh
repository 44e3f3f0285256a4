// Grid-wide barrier for persistent (cooperatively launched) kernels.
//
// Arrival is one release-reduction per block on a 64-bit counter; barrier r of
// a launch waits until the counter reaches nb*(r+1).  No block resets anything
// mid-launch, so a barrier costs one reduction plus the poll that sees the last
// arrival.  Every block calls leave() once on its way out (on every path); the
// last block to leave zeroes the counter and the leave count, so the next
// launch, whatever its grid size, starts from zero.
//
// Every wait is bounded: a block that polls more than spin_limit times latches
// DBL_ERR_TIMEOUT in the status word and stops waiting; every loop of a
// persistent kernel checks the status after each barrier and returns, so the
// launch always ends and the host sees the timeout.
#pragma once

#include "dbl_internal.cuh"

namespace dbl {

constexpr unsigned long long kSpinLimit = 1ull << 24;  // polls of ~0.3-1 us each: seconds, not forever

struct GridBarrier {
    unsigned long long *count;          // arrivals in this launch
    unsigned int *left;                 // blocks that have finished this launch
    unsigned long long *trace = nullptr;  // optional phase trace: [0] marks, [1..63] %globaltimer
    unsigned long long spin_limit = kSpinLimit;  // polls before a wait gives up
};

constexpr int kTraceWords = 64;

// Barrier words inside a d_counts array (kCntBarLeft, kCntBarCount: 8-byte aligned).
inline GridBarrier grid_barrier_at(uint32_t *counts)
{
    return GridBarrier{reinterpret_cast<unsigned long long *>(counts + kCntBarCount), counts + kCntBarLeft, nullptr,
                       kSpinLimit};
}

// Threads per block of the persistent kernels: one block per SM.  Records of
// 8 words per direction need more than 64 registers a thread, so those
// kernels run 512 threads.
__host__ __device__ constexpr int pblock_of(int hs) { return hs >= 8 ? 512 : 1024; }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p)
{
    return *(const volatile uint32_t *)p;
}

// Per-thread view of the barrier for one launch (every thread keeps the same
// barrier index; only thread 0 of a block touches the counter).
struct GridSync {
    GridBarrier b;
    unsigned long long passed = 0;

    // Block 0's thread 0 records the launch start and every barrier it passes
    // in the trace (if any): where a persistent launch spends its time.
    __device__ explicit GridSync(const GridBarrier &bar) : b(bar) { mark(); }

    __device__ __forceinline__ void mark()
    {
        if (b.trace && blockIdx.x == 0 && threadIdx.x == 0 && passed + 1 < (unsigned long long)kTraceWords) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            b.trace[1 + passed] = t;
            b.trace[0] = passed + 1;
        }
    }

    // All blocks of the grid meet here.  Returns false if this block gave up.
    __device__ __forceinline__ bool sync(uint32_t *status)
    {
        __shared__ int ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            ok = 1;
            __threadfence();
            red_release_add(b.count, 1ull);
            const unsigned long long target = (unsigned long long)gridDim.x * (passed + 1);
            unsigned long long spins = 0;
            while (ld_acquire_u64(b.count) < target) {
                if (++spins > b.spin_limit) {
                    atomicCAS(status, 0u, (uint32_t)DBL_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            __threadfence();
        }
        ++passed;
        mark();
        __syncthreads();
        return ok != 0;
    }

    // Called once by every block when it is done with the barrier.
    __device__ __forceinline__ void leave()
    {
        ++passed;
        mark();  // the end of the launch, as seen by block 0
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(b.left, 1u) == gridDim.x - 1) {
                // every block has left: nobody reads the counter any more
                *(volatile unsigned long long *)b.count = 0;
                *(volatile unsigned int *)b.left = 0;
            }
        }
    }
};

}  // namespace dbl
