// Edge insertion that allocates no memory (dbl_insert_edges_noalloc).
//
// dbl_insert_edges allocates its per-edge scratch (each edge's rank among the
// edges of its source and of its destination in the batch, 8 bytes per edge)
// from the index's allocator when a batch is larger than any before it.  Some
// callers cannot allocate device memory at that point: a process whose device
// memory is already fully handed to its own pool allocator (a serving process
// that sized its pool to the whole GPU at start-up), or a latency-bound loop
// that must not wait on an allocator.  This variant takes that scratch from a
// fixed array in the library's device memory instead; everything else it uses
// was allocated when the index was built.
#include <mutex>
#include <string>

#include "dbl_internal.cuh"

namespace dbl {

// Largest batch the variant accepts, and its scratch: [rank in source batch |
// rank in destination batch], 2 x 2^20 int32 = 8 MiB.  Every GPU that loads
// the library holds this array until the process exits.
constexpr int64_t kNoAllocMaxBatch = 1 << 20;
static __device__ __align__(256) int32_t g_noalloc_scratch[2 * kNoAllocMaxBatch];

// Device address of the array, looked up once per device.  In host code the
// array's name is only a host-side stand-in, so it is never passed to a kernel.
// The address belongs to the device's primary context as it was at the first
// call: a process that resets the device (cudaDeviceReset) and goes on
// computing gets a new context, where the module may load elsewhere, so such
// a process must not call this entry point after the reset.
constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static int32_t *g_scratch_addr[kMaxDevices];

static dbl_status scratch_address(dbl_index *ix, int32_t **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_fail(ix, e, "insert_noalloc: cudaGetDevice");
    if (dev != ix->device) return fail(ix, DBL_ERR_INVALID, "insert_noalloc: the index's device is not current");
    if (dev < 0 || dev >= kMaxDevices) return fail(ix, DBL_ERR_INVALID, "insert_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e) return cuda_fail(ix, e, "insert_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = (int32_t *)p;
    }
    *out = g_scratch_addr[dev];
    return DBL_OK;
}

}  // namespace dbl

using namespace dbl;

extern "C" dbl_status dbl_insert_edges_noalloc(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b,
                                               void *stream)
{
    if (!ix) return fail(nullptr, DBL_ERR_INVALID, "index is NULL");
    if (ix->poisoned) return fail(ix, DBL_ERR_POISONED, "index poisoned by a timeout; dbl_restore it");
    if (b < 0 || (b > 0 && (!src || !dst))) return fail(ix, DBL_ERR_INVALID, "insert_noalloc: bad batch");
    if (b > kNoAllocMaxBatch)
        return fail(ix, DBL_ERR_INVALID,
                    "insert_noalloc: batch of " + std::to_string(b) + " edges exceeds the maximum of " +
                        std::to_string(kNoAllocMaxBatch) + "; split it or use dbl_insert_edges");
    if (b == 0) return DBL_OK;
    int32_t *scratch = nullptr;
    dbl_status st = scratch_address(ix, &scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = flush_insertions(ix, s))) return st;  // batches queued earlier (DBL_FLAG_DEFER) come first
    st = insert_edges_core(ix, src, dst, b, scratch, scratch + kNoAllocMaxBatch, s);
    if (st) return st;
    if (ix->opt.flags & DBL_FLAG_ASYNC) return DBL_OK;
    return read_status(ix, s);
}
