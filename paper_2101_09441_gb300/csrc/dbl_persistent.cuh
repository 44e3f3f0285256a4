// Grid-wide barrier for persistent (cooperatively launched) kernels.
//
// Every wait is bounded: a block that waits longer than kSpinLimit polls
// latches DBL_ERR_TIMEOUT in the status word and leaves the barrier; every
// loop of a persistent kernel checks the status after each barrier and
// returns, so the launch always ends and the host sees the timeout.
#pragma once

#include "dbl_internal.cuh"

namespace dbl {

struct GridBarrier {
    unsigned int *arrived;  // blocks arrived in the current phase
    unsigned int *phase;    // generation counter
};

constexpr unsigned long long kSpinLimit = 1ull << 24;  // polls of ~0.1-1 us each: seconds, not forever

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p)
{
    return *(const volatile uint32_t *)p;
}

// All blocks of the grid meet here.  Returns false if this block gave up.
__device__ __forceinline__ bool grid_sync(const GridBarrier &b, uint32_t *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned int gen = ld_acquire(b.phase);
        __threadfence();
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(b.arrived, 1u) == nb - 1) {
            *(volatile unsigned int *)b.arrived = 0;
            __threadfence();
            atomicAdd(b.phase, 1u);
        } else {
            unsigned long long spins = 0;
            while (ld_acquire(b.phase) == gen) {
                if (++spins > kSpinLimit) {
                    atomicCAS(status, 0u, (uint32_t)DBL_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace dbl
