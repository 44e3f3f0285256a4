// Writing an index to a file and reading it back (dbl_save, dbl_load).
//
// The file holds what the index's answers and later insertions depend on:
// the base graph, the landmark and leaf choices, the labels, the per-vertex
// adjacency metadata and the used part of the two inserted-edge pools, the
// vertex count and the counters of stored edges.  Loading builds the index
// around the base graph without computing labels (the same preparation as
// dbl_build: CSR-in, landmark and leaf arrays) and then puts the saved state
// in place; the allocation sizes follow from the saved capacities, so every
// pool offset in the metadata stays valid.  Snapshots are not saved.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>

#include "dbl_internal.cuh"

namespace dbl {
namespace {

constexpr char kMagic[8] = {'D', 'B', 'L', 'I', 'N', 'D', 'E', 'X'};
constexpr uint32_t kVersion = 1;
constexpr size_t kStageBytes = 64ull << 20;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t rw;  // 64-bit words per label record
    int64_t n, n_cap, n_build, m, k, kprime;
    int64_t edge_cap, slots0, pool_cap, edges_stored;
    int64_t top[2];  // used entries of the two inserted-edge pools
    int64_t reserved[4];
};

struct FileCloser {
    void operator()(FILE *f) const
    {
        if (f) std::fclose(f);
    }
};
using File = std::unique_ptr<FILE, FileCloser>;

// Device bytes through one pinned staging buffer, kStageBytes at a time.
struct Stage {
    char *h = nullptr;
    ~Stage()
    {
        if (h) cudaFreeHost(h);
    }
    bool init()
    {
        if (cudaMallocHost((void **)&h, kStageBytes) != cudaSuccess) {
            cudaGetLastError();
            h = nullptr;
        }
        return h != nullptr;
    }
};

bool write_dev(FILE *f, const void *d, size_t bytes, Stage &st, cudaStream_t s)
{
    for (size_t off = 0; off < bytes; off += kStageBytes) {
        const size_t c = std::min(kStageBytes, bytes - off);
        if (cudaMemcpyAsync(st.h, (const char *)d + off, c, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return false;
        if (std::fwrite(st.h, 1, c, f) != c) return false;
    }
    return true;
}

bool read_dev(FILE *f, void *d, size_t bytes, Stage &st, cudaStream_t s)
{
    for (size_t off = 0; off < bytes; off += kStageBytes) {
        const size_t c = std::min(kStageBytes, bytes - off);
        if (std::fread(st.h, 1, c, f) != c) return false;
        if (cudaMemcpyAsync((char *)d + off, st.h, c, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return false;
    }
    return true;
}

bool width_ok(int64_t w) { return w == 16 || w == 32 || w == 64 || w == 128 || w == 256; }

// Device buffers for the base graph and choices while the index is built.
struct Temp {
    void *p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    ~Temp()
    {
        for (void *q : p)
            if (q) cudaFree(q);
    }
};

}  // namespace
}  // namespace dbl

using namespace dbl;

dbl_status dbl_save(dbl_index *ix, const char *path, void *stream)
{
    if (!ix || !path) return fail(ix, DBL_ERR_INVALID, "save: NULL argument");
    if (ix->poisoned) return fail(ix, DBL_ERR_POISONED, "save: index poisoned; dbl_restore it");
    cudaStream_t s = (cudaStream_t)stream;
    if (dbl_status fs = flush_insertions(ix, s)) return fs;  // queued batches are part of the index
    FileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.rw = (uint32_t)ix->rw;
    h.n = ix->n;
    h.n_cap = ix->n_cap;
    h.n_build = ix->n_build;
    h.m = ix->m;
    h.k = ix->k;
    h.kprime = ix->kp;
    h.edge_cap = ix->edge_cap;
    h.slots0 = ix->slots0;
    h.pool_cap = ix->pool_cap;
    h.edges_stored = ix->edges_stored;
    if (cudaMemcpyAsync(h.top, ix->d_pool_top, sizeof(h.top), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_fail(ix, cudaGetLastError(), "save: pool tops");
    if (h.top[0] < 0 || h.top[1] < 0 || h.top[0] > h.pool_cap || h.top[1] > h.pool_cap)
        return fail(ix, DBL_ERR_INVALID, "save: pool tops out of range");
    Stage st;
    if (!st.init()) return fail(ix, DBL_ERR_OOM, "save: pinned staging buffer");
    File f(std::fopen(path, "wb"));
    if (!f) return fail(ix, DBL_ERR_IO, std::string("save: cannot open ") + path);
    const size_t nc = (size_t)ix->n_cap;
    bool ok = std::fwrite(&h, sizeof(h), 1, f.get()) == 1 &&
              write_dev(f.get(), ix->out_ptr, 4 * ((size_t)ix->n_build + 1), st, s) &&
              write_dev(f.get(), ix->out_col, 4 * (size_t)ix->m, st, s) &&
              write_dev(f.get(), ix->landmarks, 4 * (size_t)ix->k, st, s) &&
              write_dev(f.get(), ix->leaf_bucket, 4 * nc, st, s) && write_dev(f.get(), ix->leaf_role, nc, st, s) &&
              write_dev(f.get(), ix->vm, sizeof(VMeta) * nc, st, s) &&
              write_dev(f.get(), ix->rec, 8 * nc * (size_t)ix->rw, st, s) &&
              write_dev(f.get(), ix->pool_out, 4 * (size_t)h.top[0], st, s) &&
              write_dev(f.get(), ix->pool_in, 4 * (size_t)h.top[1], st, s);
    ok = (std::fflush(f.get()) == 0) && ok;
    if (!ok) {
        cudaGetLastError();
        return fail(ix, DBL_ERR_IO, std::string("save: writing ") + path + " failed");
    }
    return DBL_OK;
}

dbl_status dbl_load(const char *path, const dbl_options *opt, void *stream, dbl_index **out)
{
    if (!path || !out) return fail(nullptr, DBL_ERR_INVALID, "load: NULL argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    File f(std::fopen(path, "rb"));
    if (!f) return fail(nullptr, DBL_ERR_IO, std::string("load: cannot open ") + path);
    FileHeader h;
    if (std::fread(&h, sizeof(h), 1, f.get()) != 1 || std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 ||
        h.version != kVersion)
        return fail(nullptr, DBL_ERR_IO, std::string("load: ") + path + " is not an index file of this version");
    if (h.n < 0 || h.n_build < 0 || h.n_build > h.n || h.n > h.n_cap || h.n_cap >= (1ll << 31) || h.m < 0 ||
        h.m >= (1ll << 31) || !width_ok(h.k) || !width_ok(h.kprime) || h.top[0] < 0 || h.top[1] < 0 ||
        h.top[0] > h.pool_cap || h.top[1] > h.pool_cap || h.rw < 2 || h.rw > 16)
        return fail(nullptr, DBL_ERR_IO, std::string("load: ") + path + " has inconsistent sizes");
    Stage st;
    if (!st.init()) return fail(nullptr, DBL_ERR_OOM, "load: pinned staging buffer");
    const size_t nc = (size_t)h.n_cap, nb = (size_t)h.n_build;
    Temp t;  // base CSR, landmarks, leaf buckets and roles of the base vertices
    const size_t tb[5] = {4 * (nb + 1), 4 * (size_t)h.m + 4, 4 * (size_t)h.k, 4 * nc + 4, nc + 4};
    for (int i = 0; i < 5; ++i)
        if (cudaMalloc(&t.p[i], tb[i]) != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, DBL_ERR_OOM, "load: device staging");
        }
    if (!read_dev(f.get(), t.p[0], 4 * (nb + 1), st, s) || !read_dev(f.get(), t.p[1], 4 * (size_t)h.m, st, s) ||
        !read_dev(f.get(), t.p[2], 4 * (size_t)h.k, st, s) || !read_dev(f.get(), t.p[3], 4 * nc, st, s) ||
        !read_dev(f.get(), t.p[4], nc, st, s)) {
        cudaGetLastError();
        return fail(nullptr, DBL_ERR_IO, std::string("load: reading ") + path + " failed");
    }
    dbl_options o;
    dbl_default_options(&o);
    if (opt) o = *opt;
    o.edge_capacity = h.edge_cap;
    o.vertex_capacity = h.n_cap;
    o.initial_slots = h.slots0 > 0 ? (int32_t)h.slots0 : -1;
    dbl_graph g{(int32_t)h.n_build, h.m, (const int32_t *)t.p[0], (const int32_t *)t.p[1]};
    dbl_index *ix = nullptr;
    dbl_status stt = build_index(&g, (const int32_t *)t.p[2], (int32_t)h.k, (const int32_t *)t.p[3],
                                 (const uint8_t *)t.p[4], (int32_t)h.kprime, &o, stream, &ix, false);
    if (stt) return stt;
    if (ix->edge_cap != h.edge_cap || ix->slots0 != h.slots0 || ix->pool_cap != h.pool_cap || ix->rw != (int)h.rw) {
        dbl_destroy(ix, stream);
        return fail(nullptr, DBL_ERR_IO, "load: the file's capacities do not match this library's layout");
    }
    bool ok = cudaMemcpyAsync(ix->leaf_bucket, t.p[3], 4 * nc, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(ix->leaf_role, t.p[4], nc, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              read_dev(f.get(), ix->vm, sizeof(VMeta) * nc, st, s) &&
              read_dev(f.get(), ix->rec, 8 * nc * (size_t)h.rw, st, s) &&
              read_dev(f.get(), ix->pool_out, 4 * (size_t)h.top[0], st, s) &&
              read_dev(f.get(), ix->pool_in, 4 * (size_t)h.top[1], st, s) &&
              cudaMemcpyAsync(ix->d_pool_top, h.top, sizeof(h.top), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemsetAsync(ix->dirty, 0, 4 * (size_t)ix->dirty_words, s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess;  // h.top lives on this stack frame
    if (!ok) {
        cudaGetLastError();
        dbl_destroy(ix, stream);
        return fail(nullptr, DBL_ERR_IO, std::string("load: reading ") + path + " failed");
    }
    ix->n = (int32_t)h.n;
    ix->edges_stored = h.edges_stored;
    *out = ix;
    return DBL_OK;
}
