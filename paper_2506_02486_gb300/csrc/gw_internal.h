// gw_internal.h -- host-side objects behind the gbwave C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "gbwave.h"
#include "gw_device.h"
#include "gw_kernels.h"
#include "stream_pool.h"

namespace gw {

// thread-local error message; returns `code` for tail calls
gw_status fail(gw_status code, const char *fmt, ...);
gw_status cuda_fail(cudaError_t e, const char *what);

#define GW_TRY_CUDA(call)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::gw::cuda_fail(e_, #call); \
    } while (0)

#define GW_TRY(call)                    \
    do {                                \
        gw_status s_ = (call);          \
        if (s_ != GW_OK) return s_;     \
    } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// CUDA streams for the stream pool: non-blocking (no implicit order with the
// legacy default stream), created on the context's device.
struct CudaStreams {
    using Handle = cudaStream_t;
    gw_status create(Handle *h)
    {
        cudaError_t e = cudaStreamCreateWithFlags(h, cudaStreamNonBlocking);
        return e == cudaSuccess ? GW_OK : cuda_fail(e, "pool stream create");
    }
    gw_status done(Handle h, bool *d)
    {
        cudaError_t e = cudaStreamQuery(h);
        if (e == cudaErrorNotReady) {
            (void)cudaGetLastError();   // not an error: still running
            *d = false;
            return GW_OK;
        }
        *d = e == cudaSuccess;
        return e == cudaSuccess ? GW_OK : cuda_fail(e, "pool stream query");
    }
    gw_status sync(Handle h)
    {
        cudaError_t e = cudaStreamSynchronize(h);
        return e == cudaSuccess ? GW_OK : cuda_fail(e, "pool stream sync");
    }
    void destroy(Handle h) { cudaStreamDestroy(h); }
};

// One global allocation (paper section 3.2).
struct Alloc {
    bool symmetric = true;
    size_t off = 0;             // symmetric: offset in every rank segment
    size_t bytes = 0;           // symmetric: bytes per rank
    size_t rec_off = 0;         // asymmetric: symmetric 32-B record offset
    std::vector<size_t> aoff;   // asymmetric: per-rank data offset
    std::vector<size_t> abytes; // asymmetric: per-rank bytes
};

// A first-fit free list over [lo, hi) offsets with coalescing.
struct FreeList {
    std::map<size_t, size_t> blocks;   // offset -> size
    void add(size_t off, size_t size);
    bool take_low(size_t size, size_t *off);    // lowest fitting block
    bool take_high(size_t size, size_t *off);   // highest fitting block
};

}  // namespace gw

// 32-byte second-level pointer record (section 3.2), as stored in device
// memory at the symmetric record offset of each rank.
struct gw_record32 {
    uint64_t addr;
    uint64_t bytes;
    uint32_t rank;
    uint32_t flags;
    uint64_t reserved;
};
static_assert(sizeof(gw_record32) == 32, "record size");

struct gw_ctx {
    int device = -1;            // -1: host-only context
    char *base = nullptr;
    size_t bytes = 0;
    int nranks = 0;
    size_t rank_bytes = 0;
    // symmetric heap: offsets below sym_top are symmetric (same on all
    // ranks); asymmetric data of rank r lives at [asym_low[r], rank_bytes)
    size_t sym_top = 0;
    gw::FreeList sym_free;
    std::vector<size_t> asym_low;
    std::vector<gw::FreeList> asym_free;
    std::unordered_map<uint64_t, gw::Alloc> allocs;
    uint64_t next_id = 1;
    // remote pointer cache: (id, rank) -> resolved address
    std::unordered_map<uint64_t, char *> ptr_cache;
    uint64_t cache_hits = 0, cache_misses = 0;
    // streams that carried puts since the last fence
    std::vector<cudaStream_t> put_streams;
    // streams of the non-blocking puts and gets (bounded concurrency)
    gw::StreamPool<gw::CudaStreams> pool;
    std::vector<cudaEvent_t> pool_events;   // one per pool stream (joins)
    std::recursive_mutex mu;
    int num_sms = 0;
    // autotuner results: shape/split/type key -> time per step of each tile
    std::map<std::string, std::vector<double>> tuned;   // ms per tile
    // host -> device uploads of models (gw_set_model*): a copy stream and,
    // per half of the staging buffer, "copied" and "used" events
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_ev[4] = {nullptr, nullptr, nullptr, nullptr};

    char *rank_base(int r) const { return base + (size_t)r * rank_bytes; }
};

namespace gw {
// Internal allocation helpers used by domains (caller holds ctx->mu).
gw_status ctx_alloc_sym(gw_ctx *c, size_t bytes, gw_gptr *out);
gw_status ctx_alloc_asym(gw_ctx *c, const size_t *bytes, gw_gptr *out);
gw_status ctx_resolve(gw_ctx *c, gw_gptr g, int rank, char **addr,
                      size_t *bytes);
gw_status ctx_free(gw_ctx *c, gw_gptr g);
// A private block in one rank's asymmetric region (no record), used for
// per-domain metadata.  Returns its address.
gw_status ctx_alloc_local(gw_ctx *c, int rank, size_t bytes, gw_gptr *out,
                          char **addr);
}  // namespace gw
