// cannon.cpp -- the paper's matrix-multiplication workload (section 5):
// Cannon's algorithm as a ring exchange over P ranks that live in one HBM.
//
// Each rank owns, in symmetric allocations of the context's segment, its
// row stripe of A (Ns x N BF16), two B stripe buffers (Ns x N BF16, B
// column stripes stored K contiguous: the paper's extra stripe that lets
// the next stripe arrive during the product) and its row stripe of C
// (Ns x N FP32).  Step s: every rank multiplies its A stripe by the B
// stripe it holds (one launch of the tensor-core kernel for all ranks),
// while non-blocking puts on the stream pool send that stripe into the
// spare buffer of rank r - 1; a fence orders the next step after the puts.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "gw_internal.h"

using namespace gw;

struct gw_cannon {
    gw_ctx *ctx = nullptr;
    int n = 0, p = 0, ns = 0;
    gw_gptr ga = 0, gb[2] = {0, 0}, gc = 0;
    int cur = 0;              // B buffer holding the current stripes
    int off = 0;              // rank r holds B column stripe (r + off) mod p
    // A boxes of 128 and 256 rows; B boxes of 256 rows per buffer
    CUtensorMap map_a[2];
    CUtensorMap map_b[2];
    int tile_m = 256;         // rows of one CTA's output tile (128 or 256)
    int group = 4;            // tile rows per raster group
    unsigned *err = nullptr;  // device error word
    gw_gptr gerr = 0;
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double gemm_ms = 0.0;
    long long launches = 0;
    int grid = 0;
};

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// {K, rows, rank} over the stripes of one symmetric BF16 allocation; box
// 64 (one 128-byte swizzle row) x box_rows x 1; rows and K beyond the
// stripe read as zeros.
gw_status encode_stripes(gw_cannon *cn, CUtensorMap *m, gw_gptr g, int box_rows)
{
    auto fn = encoder();
    if (!fn) return fail(GW_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    char *base = nullptr;
    GW_TRY(ctx_resolve(cn->ctx, g, 0, &base, nullptr));
    cuuint64_t dims[3] = {(cuuint64_t)cn->n, (cuuint64_t)cn->ns, (cuuint64_t)cn->p};
    cuuint64_t strides[2] = {(cuuint64_t)cn->n * 2, (cuuint64_t)cn->ctx->rank_bytes};
    cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(GW_ERR_CUDA, "cuTensorMapEncodeTiled (stripes) failed (%d)", (int)r);
    return GW_OK;
}

char *rank_ptr(gw_cannon *cn, gw_gptr g, int r)
{
    char *p = nullptr;
    ctx_resolve(cn->ctx, g, r, &p, nullptr);
    return p;
}

gw_status check_err(gw_cannon *cn)
{
    unsigned e = 0;
    GW_TRY_CUDA(cudaMemcpy(&e, cn->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e & ERRB_TIMEOUT)
        return fail(GW_ERR_TIMEOUT, "a tensor-core kernel wait gave up (error bits 0x%x)", e);
    if (e) return fail(GW_ERR_STATE, "device error bits 0x%x", e);
    return GW_OK;
}

// One step: the block products of every rank with the stripes it holds.
// skip_loads / wait_ns: the bounded-wait self-test.
gw_status launch_step(gw_cannon *cn, cudaStream_t s, int skip_loads = 0,
                      unsigned long long wait_ns = kWaitLimitNsHost)
{
    GemmArgs a;
    std::memset(&a, 0, sizeof a);
    a.nprob = cn->p;
    a.k = cn->n;
    a.m = cn->ns;
    a.n = cn->ns;
    // C stripes: rank r's block at rank r's C base, columns of stripe j;
    // offsets are taken from rank 0's stripe
    char *c0 = rank_ptr(cn, cn->gc, 0);
    for (int r = 0; r < cn->p; ++r) {
        const int j = (r + cn->off) % cn->p;
        a.a_rank[r] = r;
        a.b_rank[r] = r;
        const long long rank_off = (long long)(rank_ptr(cn, cn->gc, r) - c0) / 4;
        a.c_off[r] = rank_off + (long long)j * cn->ns;
    }
    a.c = reinterpret_cast<float *>(c0);
    a.ldc = cn->n;
    a.group = cn->group;
    a.err = cn->err;
    a.wait_ns = wait_ns;
    a.skip_loads = skip_loads;
    if (cn->timing) GW_TRY_CUDA(cudaEventRecord(cn->ev0, s));
    GW_TRY_CUDA(launch_gemm_bf16(&cn->map_a[cn->tile_m == 256 ? 1 : 0], &cn->map_b[cn->cur],
                                 a, cn->tile_m, cn->grid, s));
    if (cn->timing) {
        GW_TRY_CUDA(cudaEventRecord(cn->ev1, s));
        GW_TRY_CUDA(cudaEventSynchronize(cn->ev1));
        float ms = 0.f;
        GW_TRY_CUDA(cudaEventElapsedTime(&ms, cn->ev0, cn->ev1));
        cn->gemm_ms += ms;
    }
    ++cn->launches;
    return GW_OK;
}

// One resident CTA per SM, never more CTAs than tiles.
gw_status set_grid(gw_cannon *cn, int tile_m)
{
    const int tm = (cn->ns + tile_m - 1) / tile_m;
    const int tn = (cn->ns + gemm_tile_n() - 1) / gemm_tile_n();
    const int tiles = cn->p * tm * tn;
    const int most = gemm_max_ctas(tile_m, cn->ctx->num_sms);
    if (most < 1) return fail(GW_ERR_CUDA, "the block-product kernel cannot be resident");
    cn->tile_m = tile_m;
    cn->grid = std::min(most, tiles);
    return GW_OK;
}

}  // namespace

extern "C" {

gw_status gw_cannon_bytes(int n, int p, size_t *per_rank)
{
    if (!per_rank || n <= 0 || p <= 0 || p > kGemmMaxProb || n % p || (n / p) == 0)
        return fail(GW_ERR_ARG, "need 1 <= P <= %d and N a positive multiple of P",
                    kGemmMaxProb);
    const size_t ns = (size_t)(n / p);
    const size_t stripe = align_up(ns * (size_t)n * 2, kAlign);
    *per_rank = 3 * stripe + align_up(ns * (size_t)n * 4, kAlign) + kAlign;
    return GW_OK;
}

gw_status gw_cannon_create(gw_ctx *c, int n, int p, gw_cannon **out)
{
    if (!c || !out) return fail(GW_ERR_ARG, "NULL argument");
    *out = nullptr;
    size_t need = 0;
    GW_TRY(gw_cannon_bytes(n, p, &need));
    if (n % 8) return fail(GW_ERR_ALIGN, "N must be a multiple of 8 (16-byte rows), got %d", n);
    if (c->device < 0) return fail(GW_ERR_STATE, "the ring needs a device context");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->nranks < p)
        return fail(GW_ERR_ARG, "the segment has %d ranks, the ring needs %d", c->nranks, p);
    GW_TRY_CUDA(cudaSetDevice(c->device));
    gw_cannon *cn = new gw_cannon();
    cn->ctx = c;
    cn->n = n;
    cn->p = p;
    cn->ns = n / p;
    const size_t stripe = (size_t)cn->ns * n;
    auto cleanup = [&](gw_status st) {
        if (cn->ga) ctx_free(c, cn->ga);
        if (cn->gb[0]) ctx_free(c, cn->gb[0]);
        if (cn->gb[1]) ctx_free(c, cn->gb[1]);
        if (cn->gc) ctx_free(c, cn->gc);
        if (cn->gerr) ctx_free(c, cn->gerr);
        if (cn->ev0) cudaEventDestroy(cn->ev0);
        if (cn->ev1) cudaEventDestroy(cn->ev1);
        delete cn;
        return st;
    };
    gw_status st = ctx_alloc_sym(c, stripe * 2, &cn->ga);
    if (st == GW_OK) st = ctx_alloc_sym(c, stripe * 2, &cn->gb[0]);
    if (st == GW_OK) st = ctx_alloc_sym(c, stripe * 2, &cn->gb[1]);
    if (st == GW_OK) st = ctx_alloc_sym(c, stripe * 4, &cn->gc);
    char *errp = nullptr;
    if (st == GW_OK) st = ctx_alloc_local(c, 0, 256, &cn->gerr, &errp);
    if (st != GW_OK) return cleanup(st);
    cn->err = reinterpret_cast<unsigned *>(errp);
    if (cudaMemset(cn->err, 0, sizeof(unsigned)) != cudaSuccess)
        return cleanup(fail(GW_ERR_CUDA, "error word"));
    for (int h = 0; h < 2 && st == GW_OK; ++h)
        st = encode_stripes(cn, &cn->map_a[h], cn->ga, 128 << h);
    for (int b = 0; b < 2 && st == GW_OK; ++b)
        st = encode_stripes(cn, &cn->map_b[b], cn->gb[b], gemm_tile_n());
    if (st != GW_OK) return cleanup(st);
    if (cudaEventCreate(&cn->ev0) != cudaSuccess || cudaEventCreate(&cn->ev1) != cudaSuccess)
        return cleanup(fail(GW_ERR_CUDA, "events"));
    st = set_grid(cn, 256);
    if (st != GW_OK) return cleanup(st);
    *out = cn;
    return GW_OK;
}

gw_status gw_cannon_schedule(gw_cannon *cn, int tile_m, int group)
{
    if (!cn) return fail(GW_ERR_ARG, "NULL argument");
    if (tile_m != 128 && tile_m != 256) return fail(GW_ERR_ARG, "tile rows must be 128 or 256");
    if (group < 1 || group > 1024) return fail(GW_ERR_ARG, "group must be in 1 .. 1024");
    std::lock_guard<std::recursive_mutex> lk(cn->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(cn->ctx->device));
    GW_TRY(set_grid(cn, tile_m));
    cn->group = group;
    return GW_OK;
}

gw_status gw_cannon_destroy(gw_cannon *cn)
{
    if (!cn) return GW_OK;
    gw_ctx *c = cn->ctx;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    ctx_free(c, cn->ga);
    ctx_free(c, cn->gb[0]);
    ctx_free(c, cn->gb[1]);
    ctx_free(c, cn->gc);
    ctx_free(c, cn->gerr);
    cudaEventDestroy(cn->ev0);
    cudaEventDestroy(cn->ev1);
    delete cn;
    return GW_OK;
}

gw_status gw_cannon_set(gw_cannon *cn, const void *a, const void *bt, int on_device)
{
    if (!cn || !a || !bt) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(cn->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(cn->ctx->device));
    const size_t sb = (size_t)cn->ns * cn->n * 2;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int r = 0; r < cn->p; ++r) {
        GW_TRY_CUDA(cudaMemcpy(rank_ptr(cn, cn->ga, r),
                               static_cast<const char *>(a) + r * sb, sb, kind));
        GW_TRY_CUDA(cudaMemcpy(rank_ptr(cn, cn->gb[0], r),
                               static_cast<const char *>(bt) + r * sb, sb, kind));
    }
    cn->cur = 0;
    cn->off = 0;
    return GW_OK;
}

gw_status gw_cannon_run(gw_cannon *cn, gw_stream stream)
{
    if (!cn) return fail(GW_ERR_ARG, "NULL argument");
    gw_ctx *c = cn->ctx;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    GW_TRY_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t sb = (size_t)cn->ns * cn->n * 2;
    for (int step = 0; step < cn->p; ++step) {
        const bool more = step + 1 < cn->p;
        // the stripes leave for rank r - 1 while they are multiplied here:
        // puts issued before the launch wait only for what `s` already
        // holds (the previous step, which read the buffers they overwrite)
        if (more)
            for (int r = 0; r < cn->p; ++r)
                GW_TRY(gw_put_nbi(c, cn->gb[cn->cur ^ 1], (r + cn->p - 1) % cn->p, 0,
                                  rank_ptr(cn, cn->gb[cn->cur], r), sb, stream));
        GW_TRY(launch_step(cn, s));
        if (more) {
            GW_TRY(gw_fence(c, stream));
            cn->cur ^= 1;
            cn->off = (cn->off + 1) % cn->p;
        }
    }
    return GW_OK;
}

gw_status gw_cannon_read_c(gw_cannon *cn, void *out, int on_device)
{
    if (!cn || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(cn->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(cn->ctx->device));
    GW_TRY_CUDA(cudaDeviceSynchronize());
    GW_TRY(check_err(cn));
    const size_t sb = (size_t)cn->ns * cn->n * 4;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int r = 0; r < cn->p; ++r)
        GW_TRY_CUDA(cudaMemcpy(static_cast<char *>(out) + r * sb,
                               rank_ptr(cn, cn->gc, r), sb, kind));
    return GW_OK;
}

gw_status gw_cannon_sync(gw_cannon *cn)
{
    if (!cn) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(cn->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(cn->ctx->device));
    GW_TRY_CUDA(cudaDeviceSynchronize());
    return check_err(cn);
}

gw_status gw_cannon_selftest_timeout(gw_cannon *cn, unsigned limit_us, int *expired)
{
    if (!cn || !expired) return fail(GW_ERR_ARG, "NULL argument");
    if (limit_us == 0 || limit_us > 2000000u) return fail(GW_ERR_ARG, "limit must be 1 us .. 2 s");
    std::lock_guard<std::recursive_mutex> lk(cn->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(cn->ctx->device));
    GW_TRY_CUDA(cudaDeviceSynchronize());
    GW_TRY_CUDA(cudaMemset(cn->err, 0, sizeof(unsigned)));
    const bool timing = cn->timing;
    cn->timing = false;
    gw_status st = launch_step(cn, nullptr, 1, (unsigned long long)limit_us * 1000ull);
    cn->timing = timing;
    GW_TRY(st);
    GW_TRY_CUDA(cudaDeviceSynchronize());
    unsigned e = 0;
    GW_TRY_CUDA(cudaMemcpy(&e, cn->err, sizeof e, cudaMemcpyDeviceToHost));
    GW_TRY_CUDA(cudaMemset(cn->err, 0, sizeof(unsigned)));
    *expired = (e & ERRB_TIMEOUT) ? 1 : 0;
    if (*expired) return fail(GW_ERR_TIMEOUT, "block-product waits gave up as intended");
    return GW_OK;
}

gw_status gw_cannon_timing(gw_cannon *cn, int enable)
{
    if (!cn) return fail(GW_ERR_ARG, "NULL argument");
    cn->timing = enable != 0;
    cn->gemm_ms = 0.0;
    cn->launches = 0;
    return GW_OK;
}

gw_status gw_cannon_stats(gw_cannon *cn, double *gemm_ms, long long *launches, int *grid)
{
    if (!cn) return fail(GW_ERR_ARG, "NULL argument");
    if (gemm_ms) *gemm_ms = cn->gemm_ms;
    if (launches) *launches = cn->launches;
    if (grid) *grid = cn->grid;
    return GW_OK;
}

}  // extern "C"
