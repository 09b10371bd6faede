// api_segment.cpp -- errors, contexts, the global segment and PGAS
// allocation: symmetric blocks, asymmetric blocks behind 32-byte
// second-level pointers, the remote pointer cache, put/get and fence
// (paper section 3.2; Listing 1 of section 4.5 for put + fence).
#include <cstdio>
#include <cstring>

#include "gw_internal.h"

namespace gw {

static thread_local std::string t_err;

gw_status fail(gw_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

gw_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(GW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- free list

void FreeList::add(size_t off, size_t size)
{
    auto it = blocks.emplace(off, size).first;
    // merge with the next block
    auto nx = std::next(it);
    if (nx != blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        blocks.erase(nx);
    }
    // merge with the previous block
    if (it != blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            blocks.erase(it);
        }
    }
}

bool FreeList::take_low(size_t size, size_t *off)
{
    for (auto it = blocks.begin(); it != blocks.end(); ++it) {
        if (it->second >= size) {
            *off = it->first;
            size_t rest = it->second - size;
            size_t roff = it->first + size;
            blocks.erase(it);
            if (rest) blocks.emplace(roff, rest);
            return true;
        }
    }
    return false;
}

bool FreeList::take_high(size_t size, size_t *off)
{
    for (auto it = blocks.rbegin(); it != blocks.rend(); ++it) {
        if (it->second >= size) {
            size_t boff = it->first, bsz = it->second;
            *off = boff + bsz - size;
            blocks.erase(std::next(it).base());
            if (bsz > size) blocks.emplace(boff, bsz - size);
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------- allocation

static size_t min_asym_low(const gw_ctx *c)
{
    size_t m = c->rank_bytes;
    for (size_t v : c->asym_low) m = v < m ? v : m;
    return m;
}

gw_status ctx_alloc_sym(gw_ctx *c, size_t bytes, gw_gptr *out)
{
    if (!c->base) return fail(GW_ERR_STATE, "no segment attached");
    size_t sz = align_up(bytes ? bytes : 1, kAlign);
    size_t off;
    if (!c->sym_free.take_low(sz, &off)) {
        if (c->sym_top + sz > min_asym_low(c))
            return fail(GW_ERR_BUDGET,
                        "symmetric allocation of %zu bytes does not fit "
                        "(used %zu of %zu per rank)", sz, c->sym_top,
                        c->rank_bytes);
        off = c->sym_top;
        c->sym_top += sz;
    }
    Alloc a;
    a.symmetric = true;
    a.off = off;
    a.bytes = sz;
    uint64_t id = c->next_id++;
    c->allocs[id] = a;
    *out = id;
    return GW_OK;
}

static gw_status write_record(gw_ctx *c, int r, size_t rec_off,
                              const gw_record32 &rec)
{
    char *dst = c->rank_base(r) + rec_off;
    if (c->device < 0) {
        std::memcpy(dst, &rec, sizeof rec);
        return GW_OK;
    }
    GW_TRY_CUDA(cudaMemcpy(dst, &rec, sizeof rec, cudaMemcpyHostToDevice));
    return GW_OK;
}

static gw_status alloc_asym_impl(gw_ctx *c, const size_t *bytes,
                                 bool with_record, gw_gptr *out)
{
    if (!c->base) return fail(GW_ERR_STATE, "no segment attached");
    Alloc a;
    a.symmetric = false;
    a.aoff.assign(c->nranks, 0);
    a.abytes.assign(c->nranks, 0);
    gw_gptr rec_id = 0;
    if (with_record) {
        // the second-level pointer itself is a symmetric 32-byte block
        GW_TRY(ctx_alloc_sym(c, sizeof(gw_record32), &rec_id));
        a.rec_off = c->allocs[rec_id].off;
    }
    std::vector<int> done;
    for (int r = 0; r < c->nranks; ++r) {
        size_t sz = align_up(bytes[r], kAlign);
        if (sz == 0) continue;
        size_t off;
        if (!c->asym_free[r].take_high(sz, &off)) {
            if (c->asym_low[r] < c->sym_top + sz) {
                for (int q : done) c->asym_free[q].add(a.aoff[q], a.abytes[q]);
                if (rec_id) ctx_free(c, rec_id);
                return fail(GW_ERR_BUDGET,
                            "asymmetric allocation of %zu bytes on rank %d "
                            "does not fit", sz, r);
            }
            c->asym_low[r] -= sz;
            off = c->asym_low[r];
        }
        a.aoff[r] = off;
        a.abytes[r] = sz;
        done.push_back(r);
    }
    if (rec_id) {
        // the record allocation is owned by this allocation now
        c->allocs.erase(rec_id);
        for (int r = 0; r < c->nranks; ++r) {
            gw_record32 rec{};
            rec.addr = a.abytes[r] ? (uint64_t)(uintptr_t)(c->rank_base(r) + a.aoff[r]) : 0;
            rec.bytes = a.abytes[r];
            rec.rank = (uint32_t)r;
            rec.flags = 1;
            GW_TRY(write_record(c, r, a.rec_off, rec));
        }
    } else {
        a.rec_off = SIZE_MAX;
    }
    uint64_t id = c->next_id++;
    c->allocs[id] = a;
    *out = id;
    return GW_OK;
}

gw_status ctx_alloc_asym(gw_ctx *c, const size_t *bytes, gw_gptr *out)
{
    return alloc_asym_impl(c, bytes, true, out);
}

gw_status ctx_alloc_local(gw_ctx *c, int rank, size_t bytes, gw_gptr *out,
                          char **addr)
{
    if (rank < 0 || rank >= c->nranks) return fail(GW_ERR_ARG, "bad rank");
    std::vector<size_t> b(c->nranks, 0);
    b[rank] = bytes ? bytes : 1;
    GW_TRY(alloc_asym_impl(c, b.data(), false, out));
    *addr = c->rank_base(rank) + c->allocs[*out].aoff[rank];
    return GW_OK;
}

static void release_sym(gw_ctx *c, size_t off, size_t sz)
{
    c->sym_free.add(off, sz);
    // shrink the symmetric top if the highest free block reaches it
    while (!c->sym_free.blocks.empty()) {
        auto last = std::prev(c->sym_free.blocks.end());
        if (last->first + last->second != c->sym_top) break;
        c->sym_top = last->first;
        c->sym_free.blocks.erase(last);
    }
}

static void release_asym(gw_ctx *c, int r, size_t off, size_t sz)
{
    c->asym_free[r].add(off, sz);
    while (!c->asym_free[r].blocks.empty()) {
        auto first = c->asym_free[r].blocks.begin();
        if (first->first != c->asym_low[r]) break;
        c->asym_low[r] = first->first + first->second;
        c->asym_free[r].blocks.erase(first);
    }
}

gw_status ctx_free(gw_ctx *c, gw_gptr g)
{
    auto it = c->allocs.find(g);
    if (it == c->allocs.end()) return fail(GW_ERR_ARG, "unknown allocation");
    Alloc a = it->second;
    c->allocs.erase(it);
    if (a.symmetric) {
        release_sym(c, a.off, a.bytes);
    } else {
        for (int r = 0; r < c->nranks; ++r)
            if (a.abytes[r]) release_asym(c, r, a.aoff[r], a.abytes[r]);
        if (a.rec_off != SIZE_MAX)
            release_sym(c, a.rec_off, align_up(sizeof(gw_record32), kAlign));
    }
    // cache entries of this allocation are no longer valid
    for (int r = 0; r < c->nranks; ++r) c->ptr_cache.erase((g << 16) | (uint64_t)r);
    return GW_OK;
}

gw_status ctx_resolve(gw_ctx *c, gw_gptr g, int rank, char **addr,
                      size_t *bytes)
{
    auto it = c->allocs.find(g);
    if (it == c->allocs.end()) return fail(GW_ERR_ARG, "unknown allocation");
    if (rank < 0 || rank >= c->nranks) return fail(GW_ERR_ARG, "bad rank %d", rank);
    const Alloc &a = it->second;
    if (a.symmetric) {
        // offset translation: the same offset in the target rank's segment
        *addr = c->rank_base(rank) + a.off;
        if (bytes) *bytes = a.bytes;
        return GW_OK;
    }
    if (a.rec_off == SIZE_MAX) {
        *addr = a.abytes[rank] ? c->rank_base(rank) + a.aoff[rank] : nullptr;
        if (bytes) *bytes = a.abytes[rank];
        return GW_OK;
    }
    uint64_t key = (g << 16) | (uint64_t)rank;
    auto hit = c->ptr_cache.find(key);
    if (hit != c->ptr_cache.end()) {
        ++c->cache_hits;
        *addr = hit->second;
        if (bytes) *bytes = a.abytes[rank];
        return GW_OK;
    }
    // two-step access: fetch the second-level pointer, then use it
    ++c->cache_misses;
    gw_record32 rec{};
    const char *src = c->rank_base(rank) + a.rec_off;
    if (c->device < 0)
        std::memcpy(&rec, src, sizeof rec);
    else
        GW_TRY_CUDA(cudaMemcpy(&rec, src, sizeof rec, cudaMemcpyDeviceToHost));
    if (rec.rank != (uint32_t)rank || rec.bytes != a.abytes[rank])
        return fail(GW_ERR_STATE, "corrupt second-level pointer record");
    char *p = reinterpret_cast<char *>((uintptr_t)rec.addr);
    c->ptr_cache[key] = p;
    *addr = p;
    if (bytes) *bytes = rec.bytes;
    return GW_OK;
}

}  // namespace gw

using namespace gw;

// ================================================================ C ABI

extern "C" {

const char *gw_last_error(void) { return t_err.c_str(); }

const char *gw_status_string(gw_status s)
{
    switch (s) {
    case GW_OK: return "GW_OK";
    case GW_ERR_ARG: return "GW_ERR_ARG";
    case GW_ERR_BUDGET: return "GW_ERR_BUDGET";
    case GW_ERR_ALIGN: return "GW_ERR_ALIGN";
    case GW_ERR_CUDA: return "GW_ERR_CUDA";
    case GW_ERR_TIMEOUT: return "GW_ERR_TIMEOUT";
    case GW_ERR_STATE: return "GW_ERR_STATE";
    case GW_ERR_NUMERIC: return "GW_ERR_NUMERIC";
    case GW_ERR_NOMEM: return "GW_ERR_NOMEM";
    default: return "GW_ERR_UNKNOWN";
    }
}

const char *gw_version(void) { return "gbwave 0.1 (sm_103a)"; }

gw_status gw_ctx_create(gw_ctx **out, int device)
{
    if (!out) return fail(GW_ERR_ARG, "out is NULL");
    *out = nullptr;
    gw_ctx *c = new (std::nothrow) gw_ctx();
    if (!c) return fail(GW_ERR_NOMEM, "out of host memory");
    c->device = device < 0 ? -1 : device;
    if (device >= 0) {
        int n = 0;
        cudaError_t e = cudaGetDeviceCount(&n);
        if (e != cudaSuccess || device >= n) {
            delete c;
            return e != cudaSuccess ? cuda_fail(e, "cudaGetDeviceCount")
                                    : fail(GW_ERR_ARG, "no CUDA device %d", device);
        }
        e = cudaSetDevice(device);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaSetDevice");
        }
    }
    *out = c;
    return GW_OK;
}

gw_status gw_ctx_destroy(gw_ctx *c)
{
    if (!c) return GW_OK;
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        c->pool.destroy();      // streams with pending work finish first
        for (cudaEvent_t ev : c->pool_events) cudaEventDestroy(ev);
        if (c->up_stream) {
            cudaStreamSynchronize(c->up_stream);
            cudaStreamDestroy(c->up_stream);
        }
        for (cudaEvent_t ev : c->up_ev)
            if (ev) cudaEventDestroy(ev);
    }
    delete c;
    return GW_OK;
}

gw_status gw_segment_attach(gw_ctx *c, void *base, size_t bytes, int nranks,
                            int zero)
{
    if (!c || !base || nranks <= 0) return fail(GW_ERR_ARG, "bad segment arguments");
    if (reinterpret_cast<uintptr_t>(base) % kAlign)
        return fail(GW_ERR_ALIGN, "segment base must be %zu-byte aligned", kAlign);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->base) return fail(GW_ERR_STATE, "segment already attached");
    size_t rb = bytes / (size_t)nranks / 4096 * 4096;
    if (rb < 4096) return fail(GW_ERR_BUDGET, "segment too small for %d ranks", nranks);
    if (c->device >= 0 && zero) {
        GW_TRY_CUDA(cudaSetDevice(c->device));
        GW_TRY_CUDA(cudaMemset(base, 0, rb * nranks));
    }
    c->base = static_cast<char *>(base);
    c->bytes = bytes;
    c->nranks = nranks;
    c->rank_bytes = rb;
    c->sym_top = 0;
    c->asym_low.assign(nranks, rb);
    c->asym_free.assign(nranks, FreeList());
    return GW_OK;
}

gw_status gw_segment_info(gw_ctx *c, size_t *rank_bytes, size_t *sym_used,
                          size_t *asym_used)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (rank_bytes) *rank_bytes = c->rank_bytes;
    if (sym_used) *sym_used = c->sym_top;
    if (asym_used) *asym_used = c->rank_bytes - min_asym_low(c);
    return GW_OK;
}

gw_status gw_alloc_symmetric(gw_ctx *c, size_t bytes, gw_gptr *out)
{
    if (!c || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    return ctx_alloc_sym(c, bytes, out);
}

gw_status gw_alloc_asymmetric(gw_ctx *c, const size_t *bytes, gw_gptr *out)
{
    if (!c || !out || !bytes) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    return ctx_alloc_asym(c, bytes, out);
}

gw_status gw_free(gw_ctx *c, gw_gptr g)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    return ctx_free(c, g);
}

gw_status gw_resolve(gw_ctx *c, gw_gptr g, int rank, void **addr, size_t *bytes)
{
    if (!c || !addr) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char *p = nullptr;
    GW_TRY(ctx_resolve(c, g, rank, &p, bytes));
    *addr = p;
    return GW_OK;
}

gw_status gw_ptr_cache_stats(gw_ctx *c, uint64_t *hits, uint64_t *misses)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (hits) *hits = c->cache_hits;
    if (misses) *misses = c->cache_misses;
    return GW_OK;
}

static gw_status remote_copy(gw_ctx *c, gw_gptr g, int rank, size_t off,
                             size_t bytes, char **remote)
{
    size_t sz = 0;
    char *p = nullptr;
    GW_TRY(ctx_resolve(c, g, rank, &p, &sz));
    if (off > sz || bytes > sz - off)
        return fail(GW_ERR_ARG, "range [%zu, %zu) outside the %zu-byte block",
                    off, off + bytes, sz);
    *remote = p + off;
    return GW_OK;
}

static void note_stream(gw_ctx *c, cudaStream_t s)
{
    for (cudaStream_t q : c->put_streams)
        if (q == s) return;
    c->put_streams.push_back(s);
}

gw_status gw_put(gw_ctx *c, gw_gptr dst, int dst_rank, size_t dst_off,
                 const void *src, size_t bytes, gw_stream stream)
{
    if (!c || (!src && bytes)) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char *p = nullptr;
    GW_TRY(remote_copy(c, dst, dst_rank, dst_off, bytes, &p));
    if (!bytes) return GW_OK;
    if (c->device < 0) {
        std::memcpy(p, src, bytes);
        return GW_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GW_TRY_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToDevice, s));
    note_stream(c, s);
    return GW_OK;
}

gw_status gw_get(gw_ctx *c, void *dst, gw_gptr src, int src_rank,
                 size_t src_off, size_t bytes, gw_stream stream)
{
    if (!c || (!dst && bytes)) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char *p = nullptr;
    GW_TRY(remote_copy(c, src, src_rank, src_off, bytes, &p));
    if (!bytes) return GW_OK;
    if (c->device < 0) {
        std::memcpy(dst, p, bytes);
        return GW_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GW_TRY_CUDA(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyDeviceToDevice, s));
    note_stream(c, s);
    return GW_OK;
}

gw_status gw_fence(gw_ctx *c, gw_stream stream)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->device < 0) {
        c->put_streams.clear();
        return GW_OK;
    }
    cudaStream_t target = static_cast<cudaStream_t>(stream);
    // join every stream that carried puts into the target stream
    for (cudaStream_t s : c->put_streams) {
        if (s == target) continue;
        cudaEvent_t ev;
        GW_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(target, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return cuda_fail(e, "fence join");
    }
    c->put_streams.clear();
    // and every pool stream with an unreleased operation; joined streams are
    // released (work issued on them later is ordered after the join anyway)
    const std::vector<int> &act = c->pool.active();
    for (int idx : act) {
        cudaEvent_t ev = c->pool_events[idx];
        GW_TRY_CUDA(cudaEventRecord(ev, c->pool.handle(idx)));
        GW_TRY_CUDA(cudaStreamWaitEvent(target, ev, 0));
    }
    if (!act.empty()) c->pool.count_fence();
    c->pool.release_all();
    return GW_OK;
}

// One copy on a pool stream, after the work already on `after`.
static gw_status pool_copy(gw_ctx *c, void *dst, const void *src, size_t bytes,
                           cudaStream_t after)
{
    GW_TRY_CUDA(cudaSetDevice(c->device));
    int idx = -1;
    GW_TRY(c->pool.acquire(&idx));
    while ((int)c->pool_events.size() <= idx) {
        cudaEvent_t ev;
        GW_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->pool_events.push_back(ev);
    }
    cudaStream_t ps = c->pool.handle(idx);
    cudaEvent_t ev = c->pool_events[idx];
    GW_TRY_CUDA(cudaEventRecord(ev, after));
    GW_TRY_CUDA(cudaStreamWaitEvent(ps, ev, 0));
    GW_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ps));
    return GW_OK;
}

gw_status gw_put_nbi(gw_ctx *c, gw_gptr dst, int dst_rank, size_t dst_off,
                     const void *src, size_t bytes, gw_stream after)
{
    if (!c || (!src && bytes)) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char *p = nullptr;
    GW_TRY(remote_copy(c, dst, dst_rank, dst_off, bytes, &p));
    if (!bytes) return GW_OK;
    if (c->device < 0) {
        std::memcpy(p, src, bytes);
        return GW_OK;
    }
    return pool_copy(c, p, src, bytes, static_cast<cudaStream_t>(after));
}

gw_status gw_get_nbi(gw_ctx *c, void *dst, gw_gptr src, int src_rank,
                     size_t src_off, size_t bytes, gw_stream after)
{
    if (!c || (!dst && bytes)) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char *p = nullptr;
    GW_TRY(remote_copy(c, src, src_rank, src_off, bytes, &p));
    if (!bytes) return GW_OK;
    if (c->device < 0) {
        std::memcpy(dst, p, bytes);
        return GW_OK;
    }
    return pool_copy(c, dst, p, bytes, static_cast<cudaStream_t>(after));
}

gw_status gw_quiet(gw_ctx *c)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->device < 0) return GW_OK;
    GW_TRY_CUDA(cudaSetDevice(c->device));
    return c->pool.quiet();
}

gw_status gw_set_max_active_streams(gw_ctx *c, int n)
{
    if (!c) return fail(GW_ERR_ARG, "ctx is NULL");
    if (n < 1 || n > 64) return fail(GW_ERR_ARG, "max active streams must be 1 .. 64, got %d", n);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    c->pool.set_max_active(n);
    return GW_OK;
}

gw_status gw_pool_stats_get(gw_ctx *c, gw_pool_stats *out)
{
    if (!c || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    *out = c->pool.stats();
    return GW_OK;
}

}  // extern "C"
