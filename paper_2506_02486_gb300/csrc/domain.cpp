// domain.cpp -- one shot decomposed into subdomains that live in one HBM:
// PGAS allocation of the fields (paper section 3.2), the halo plan of
// Listing 1 (section 4.5), TMA tensor maps, the work-item schedule, CUDA
// graph chunks of K steps, model/source/receiver set-up and host I/O.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "domain_impl.h"

using namespace gw;

namespace {

constexpr size_t kStageBytes = size_t(256) << 20;   // host<->device slabs

// FP64 host precompute of the scheme's constants (the library's own; the
// scheme is not printed in the paper).
double symbol_at_pi()
{
    const double c[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                         -1.0 / 560.0};
    double s = c[0];
    for (int m = 1; m <= 4; ++m) s += 2.0 * c[m] * ((m & 1) ? -1.0 : 1.0);
    return s;
}

double nu_limit() { return std::sqrt(4.0 / (3.0 * std::fabs(symbol_at_pi()))); }

// Cerjan factor for cell i of n with a layer of w cells and constant a.
double cerjan(int i, int n, int w, double a)
{
    int d = std::min(i, n - 1 - i);
    if (d >= w) return 1.0;
    double e = a * (double)(w - d);
    return std::exp(-e * e);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

CUtensorMapDataType tma_type(int elem_size, bool bf16)
{
    switch (elem_size) {
    case 8: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    case 4: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    default: return bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    }
}

}  // namespace


namespace {

gw_status fetch_err(gw_domain *d)
{
    unsigned e = 0;
    GW_TRY_CUDA(cudaMemcpy(&e, d->d_err, sizeof e, cudaMemcpyDeviceToHost));
    if (!e) return GW_OK;
    unsigned z = 0;
    GW_TRY_CUDA(cudaMemcpy(d->d_err, &z, sizeof z, cudaMemcpyHostToDevice));
    if (e & ERRB_TIMEOUT)
        return fail(GW_ERR_TIMEOUT, "a device wait gave up (error bits 0x%x)", e);
    if (e & ERRB_NONFINITE)
        return fail(GW_ERR_NUMERIC, "non-finite wavefield norm (error bits 0x%x)", e);
    if (e & ERRB_LOCAL_OVERFLOW)
        return fail(GW_ERR_STATE, "more than %d sources and receivers inside one work item "
                    "(error bits 0x%x)", kMaxLocal, e);
    return fail(GW_ERR_STATE, "device error bits 0x%x", e);
}

gw_status sync_dom(gw_domain *d)
{
    GW_TRY_CUDA(cudaSetDevice(d->ctx->device));
    if (d->step == 0 && !d->last) {
        // never stepped: only its own setup work (legacy stream) can be in
        // flight; other shots' launches on other streams keep running
        GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    } else {
        GW_TRY_CUDA(cudaDeviceSynchronize());
    }
    return fetch_err(d);
}

gw_status local_alloc(gw_domain *d, size_t bytes, char **p, gw_gptr *g = nullptr)
{
    gw_gptr h = 0;
    GW_TRY(ctx_alloc_local(d->ctx, 0, bytes, &h, p));
    d->allocs.push_back(h);
    d->device_bytes += align_up(bytes, kAlign);
    if (g) *g = h;
    return GW_OK;
}

void drop_alloc(gw_domain *d, gw_gptr g)
{
    if (!g) return;
    auto it = std::find(d->allocs.begin(), d->allocs.end(), g);
    if (it != d->allocs.end()) d->allocs.erase(it);
    ctx_free(d->ctx, g);
}

// Encode one 3-D tensor map over a padded field array.
gw_status encode_map(gw_domain *d, CUtensorMap *out, char *base, const SubDev &s,
                     int esize, bool bf16, int box_x, int box_y)
{
    auto fn = encode_fn();
    if (!fn) return fail(GW_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)s.px, (cuuint64_t)s.py,
                          (cuuint64_t)(s.nz + 2 * R)};
    cuuint64_t strides[2] = {(cuuint64_t)s.px * esize,
                             (cuuint64_t)s.px * s.py * esize};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(out, tma_type(esize, bf16), 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(GW_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    (void)d;
    return GW_OK;
}

void build_items(gw_domain *d)
{
    d->zc = make_items(d->subs, d->ti, d->grid, d->desc.zchunk, d->desc.schedule, d->items);
    d->nitems = (int)d->items.size();
}

void build_halo_plan(gw_domain *d)
{
    d->halo.clear();
    // the copy kernel moves rows in 16-byte units of V elements
    const long long V = 16 / d->esize();
    long long most = 0;
    for (int si = 0; si < d->nsub(); ++si) {
        const SubDev &s = d->subs[si];
        for (int f = 0; f < 6; ++f) {
            int nb = s.nbr[f];
            if (nb < 0) continue;
            long long units = (f >> 1) == 0 ? (R + V - 1) / V * s.ny * s.nz
                            : (f >> 1) == 1 ? (s.nx + V - 1) / V * R * s.nz
                                            : (s.nx + V - 1) / V * s.ny * R;
            HaloDesc h{si, nb, f, 0, 0};
            d->halo.push_back(h);
            most = std::max(most, units);
        }
    }
    d->halo_units = most;
}

gw_status plan_schedule(gw_domain *d)
{
    gw_ctx *c = d->ctx;
    int ncfg = step_cfg_count(d->dtype);
    int want = d->desc.tile > 0 ? d->desc.tile - 1 : 0;
    if (want >= ncfg) return fail(GW_ERR_ARG, "tile %d not available", d->desc.tile);
    d->cfg = want;
    step_cfg_info(d->dtype, d->cfg, &d->ti);
    bool sponge = d->desc.sponge > 0;
    int occ = step_cfg_occupancy(d->dtype, d->cfg, sponge);
    if (occ <= 0) return fail(GW_ERR_CUDA, "kernel configuration does not fit an SM");
    d->grid = std::max(1, c->num_sms * occ);
    build_items(d);
    if (d->nitems == 0) return fail(GW_ERR_ARG, "empty grid");
    d->grid = std::min(d->grid, d->nitems);
    // work items to CTAs: static round robin for an undecomposed shot
    // whose tile columns fit in one round of CTAs (items alike, and the
    // CTAs on neighbouring tiles stay in step: 512^3 1-3 % faster), dynamic
    // otherwise (640^3 6.5 %, 1200^3 27 %, 2 x 2 x 2 with fused halo puts
    // 6 % faster)
    d->dynamic = dynamic_schedule(d->desc.schedule, d->nsub(), tile_columns(d->subs, d->ti),
                                  d->grid);
    // items and the norm partials of one chunk
    if (d->g_items) drop_alloc(d, d->g_items);
    size_t ib = sizeof(Item) * d->nitems;
    size_t pb = sizeof(double) * (size_t)d->nitems * (size_t)std::max(1, d->chunk);
    char *p = nullptr;
    GW_TRY(local_alloc(d, ib + pb + kAlign, &p, &d->g_items));
    d->d_items = reinterpret_cast<Item *>(p);
    d->d_partials = reinterpret_cast<double *>(p + align_up(ib, kAlign));
    GW_TRY_CUDA(cudaMemcpy(d->d_items, d->items.data(), ib, cudaMemcpyHostToDevice));
    d->shot.first_item = 0;
    d->shot.nitems = d->nitems;
    return GW_OK;
}

// Every setup call ends here: the legacy-stream copies and kernels of the
// setup are complete when it returns, so that launches on non-blocking
// streams (which do not wait for the legacy stream) see them.
gw_status push_shot(gw_domain *d)
{
    // bounding boxes of the sources and of the receivers: items outside a
    // box skip the per-item search of that list (separate boxes, so that a
    // receiver plane far from the source does not make every item between
    // them search)
    const std::vector<int4> *lists[2] = {&d->srcs, &d->recs};
    for (int l = 0; l < 2; ++l) {
        for (int a = 0; a < 3; ++a) {
            d->shot.lo[l][a] = 1 << 30;
            d->shot.hi[l][a] = -1;
        }
        for (const int4 &q : *lists[l]) {
            const int c[3] = {q.x, q.y, q.z};
            for (int a = 0; a < 3; ++a) {
                d->shot.lo[l][a] = std::min(d->shot.lo[l][a], c[a]);
                d->shot.hi[l][a] = std::max(d->shot.hi[l][a], c[a]);
            }
        }
    }
    GW_TRY_CUDA(cudaMemcpy(d->d_shot, &d->shot, sizeof(ShotDev), cudaMemcpyHostToDevice));
    GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    return GW_OK;
}

gw_status make_maps(gw_domain *d)
{
    const int es = d->esize();
    const int hl = dtype_halo(d->dtype);
    const bool bf16 = d->dtype == DT_BF16;
    std::vector<CUtensorMap> maps((size_t)d->nsub() * kMapsPerSub);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    for (int si = 0; si < d->nsub(); ++si) {
        const SubDev &s = d->subs[si];
        CUtensorMap *m = &maps[(size_t)si * kMapsPerSub];
        int hx = d->ti.tx + 2 * hl, hy = d->ti.ty + 2 * R;
        GW_TRY(encode_map(d, &m[MAP_U0_HALO], s.u[0], s, es, bf16, hx, hy));
        GW_TRY(encode_map(d, &m[MAP_U1_HALO], s.u[1], s, es, bf16, hx, hy));
        GW_TRY(encode_map(d, &m[MAP_U0_PW], s.u[0], s, es, bf16, d->ti.tx, d->ti.ty));
        GW_TRY(encode_map(d, &m[MAP_U1_PW], s.u[1], s, es, bf16, d->ti.tx, d->ti.ty));
        // reduced storage keeps coef in FP16
        int ces = d->delta ? 2 : es;
        GW_TRY(encode_map(d, &m[MAP_COEF_PW], s.coef, s, ces, false, d->ti.tx, d->ti.ty));
        if (d->delta)
            GW_TRY(encode_map(d, &m[MAP_W_PW], s.w, s, es, bf16, d->ti.tx, d->ti.ty));
    }
    GW_TRY_CUDA(cudaMemcpy(d->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice));
    return GW_OK;
}

void destroy_graph(gw_domain *d)
{
    if (d->gexec) cudaGraphExecDestroy(d->gexec);
    d->gexec = nullptr;
}

StepArgs step_args(gw_domain *d, int k)
{
    StepArgs a{};
    a.subs = d->d_subs;
    a.shots = d->d_shot;
    a.items = d->d_items;
    a.maps = d->d_maps;
    a.partials = d->d_partials;
    a.err = d->d_err;
    a.seg_base = d->ctx->base;
    a.rank_stride = (long long)d->ctx->rank_bytes;
    a.nitems = d->nitems;
    a.k = k;
    a.symmetric = d->symmetric ? 1 : 0;
    a.fused_halo = d->desc.halo_mode == GW_HALO_FUSED ? 1 : 0;
    a.nk = 1;
    a.gbar = d->d_gbar;
    a.ctr = d->d_ctr;
    a.dynamic = d->dynamic ? 1 : 0;
    return a;
}

cudaEvent_t pool_event(gw_domain *d)
{
    if (!d->ev_pool.empty()) {
        cudaEvent_t e = d->ev_pool.back();
        d->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Enqueue nk steps (k = 0..nk-1) and the chunk end.
gw_status enqueue_chunk(gw_domain *d, int nk, cudaStream_t s, bool timed)
{
    const bool sponge = d->desc.sponge > 0;
    const bool sep = d->desc.halo_mode == GW_HALO_SEPARATE && !d->halo.empty();
    // the step kernel leaves its work-item tickets at zero after every step;
    // a launch that gave up (GW_ERR_TIMEOUT) may not, so every chunk starts
    // from zero
    GW_TRY_CUDA(cudaMemsetAsync(d->d_ctr, 0, sizeof(unsigned), s));
    if (d->desc.persistent && !sep && nk > 1) {
        // all nk steps in one launch, a device-wide barrier between steps
        GW_TRY_CUDA(cudaMemsetAsync(d->d_gbar, 0, sizeof(unsigned), s));
        StepArgs a = step_args(d, 0);
        a.nk = nk;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            e0 = pool_event(d);
            e1 = pool_event(d);
            GW_TRY_CUDA(cudaEventRecord(e0, s));
        }
        GW_TRY_CUDA(launch_step(d->dtype, d->cfg, sponge, d->grid, a, s));
        if (timed) {
            GW_TRY_CUDA(cudaEventRecord(e1, s));
            d->ev_step.push_back({e0, e1});
            d->ev_steps.push_back(nk);
        }
        GW_TRY_CUDA(launch_chunk_end(d->d_shot, 1, d->d_partials, d->nitems, nk,
                                     d->d_err, s));
        return GW_OK;
    }
    for (int k = 0; k < nk; ++k) {
        StepArgs a = step_args(d, k);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            e0 = pool_event(d);
            e1 = pool_event(d);
            GW_TRY_CUDA(cudaEventRecord(e0, s));
        }
        GW_TRY_CUDA(launch_step(d->dtype, d->cfg, sponge, d->grid, a, s));
        if (timed) {
            GW_TRY_CUDA(cudaEventRecord(e1, s));
            d->ev_step.push_back({e0, e1});
            d->ev_steps.push_back(1);
        }
        if (sep) {
            cudaEvent_t h0 = nullptr, h1 = nullptr;
            if (timed) {
                h0 = pool_event(d);
                h1 = pool_event(d);
                GW_TRY_CUDA(cudaEventRecord(h0, s));
            }
            GW_TRY_CUDA(launch_halo(d->d_halo, (int)d->halo.size(), d->halo_units,
                                    d->d_subs, d->d_step, k, d->dtype, s));
            if (timed) {
                GW_TRY_CUDA(cudaEventRecord(h1, s));
                d->ev_halo.push_back({h0, h1});
            }
        }
    }
    GW_TRY_CUDA(launch_chunk_end(d->d_shot, 1, d->d_partials, d->nitems, nk,
                                 d->d_err, s));
    return GW_OK;
}

gw_status ensure_graph(gw_domain *d)
{
    if (d->gexec) return GW_OK;
    if (!d->cap_stream)
        GW_TRY_CUDA(cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking));
    GW_TRY_CUDA(cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal));
    gw_status st = enqueue_chunk(d, d->chunk, d->cap_stream, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(d->cap_stream, &g);
    if (st != GW_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&d->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return GW_OK;
}

void harvest_events(gw_domain *d)
{
    for (size_t i = 0; i < d->ev_step.size(); ++i) {
        auto &p = d->ev_step[i];
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            d->acc_ms += ms;
            d->acc_n += i < d->ev_steps.size() ? d->ev_steps[i] : 1;
        }
        d->ev_pool.push_back(p.first);
        d->ev_pool.push_back(p.second);
    }
    for (auto &p : d->ev_halo) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess)
            d->acc_halo_ms += ms;
        d->ev_pool.push_back(p.first);
        d->ev_pool.push_back(p.second);
    }
    d->ev_step.clear();
    d->ev_steps.clear();
    d->ev_halo.clear();
}

// Dense slab staging buffer (device), allocated per call.
struct Stage {
    gw_domain *d;
    gw_gptr g = 0;
    char *p = nullptr;
    size_t bytes = 0;
    ~Stage() { if (g) drop_alloc(d, g); }
};

gw_status stage_alloc(gw_domain *d, Stage &st, size_t want, size_t plane_bytes)
{
    st.d = d;
    // at least one plane, at most kStageBytes unless a plane is larger
    st.bytes = std::max(std::min(want, kStageBytes), plane_bytes + 16);
    return local_alloc(d, st.bytes, &st.p, &st.g);
}

// Host slabs of planes through the two halves of a staging buffer: the
// copy of slab i + 1 runs on the context's copy stream while the kernels of
// slab i run on the legacy stream (pinned host memory: ~210 GB/s on GB300's
// host link, so the kernels hide behind the copies).  consume(buf, z0, z1)
// enqueues the kernels for planes [z0, z1) staged at buf.
template <class F>
gw_status upload_slabs(gw_domain *d, const Stage &st, const char *h, size_t plane_bytes,
                              F &&consume)
{
    gw_ctx *c = d->ctx;
    if (!c->up_stream) {
        GW_TRY_CUDA(cudaStreamCreateWithFlags(&c->up_stream, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->up_ev)
            GW_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const size_t half = (st.bytes - 16) / 2 / kAlign * kAlign;
    const int nz = d->desc.nz;
    const int pps = (int)std::max<size_t>(1, half / plane_bytes);
    const bool two = half >= plane_bytes;       // else one slab at a time
    for (int i = 0, z = 0; z < nz; ++i, z += pps) {
        const int zh = std::min(nz, z + pps);
        const int b = two ? (i & 1) : 0;
        char *buf = st.p + (size_t)b * half;
        cudaEvent_t copied = c->up_ev[2 * b], used = c->up_ev[2 * b + 1];
        if (i >= (two ? 2 : 1)) GW_TRY_CUDA(cudaStreamWaitEvent(c->up_stream, used, 0));
        GW_TRY_CUDA(cudaMemcpyAsync(buf, h + plane_bytes * (size_t)z,
                                    plane_bytes * (size_t)(zh - z), cudaMemcpyHostToDevice,
                                    c->up_stream));
        GW_TRY_CUDA(cudaEventRecord(copied, c->up_stream));
        GW_TRY_CUDA(cudaStreamWaitEvent(nullptr, copied, 0));
        GW_TRY(consume(buf, z, zh));
        GW_TRY_CUDA(cudaEventRecord(used, nullptr));
    }
    return GW_OK;
}

int planes_per_slab(const gw_domain *d, size_t bytes_per_elem, size_t stage)
{
    size_t plane = (size_t)d->desc.nx * d->desc.ny * bytes_per_elem;
    return (int)std::max<size_t>(1, stage / plane);
}

gw_status check_dom(gw_domain *d)
{
    if (!d) return fail(GW_ERR_ARG, "domain is NULL");
    if (d->ctx->device < 0) return fail(GW_ERR_STATE, "host-only context cannot run kernels");
    GW_TRY_CUDA(cudaSetDevice(d->ctx->device));
    return GW_OK;
}

}  // namespace

namespace gw {

long long tile_columns(const std::vector<SubDev> &subs, const TileInfo &ti)
{
    long long n = 0;
    for (const SubDev &s : subs)
        n += (long long)((s.nx + ti.tx - 1) / ti.tx) * ((s.ny + ti.ty - 1) / ti.ty);
    return n;
}

bool dynamic_schedule(int sched, int nsub, long long ncols, int grid)
{
    if (sched == GW_SCHED_STATIC) return false;
    if (sched == GW_SCHED_DYNAMIC) return true;
    return nsub > 1 || ncols > grid;
}

// Work items in z-chunk-major order (CTAs running together hold
// neighbouring columns at the same depth).
int make_items(const std::vector<SubDev> &subs, const TileInfo &ti, int grid,
               int zchunk, int sched, std::vector<Item> &items, int sub_base,
               bool tail_hidden)
{
    const int TX = ti.tx, TY = ti.ty;
    const long long ncols = tile_columns(subs, ti);
    int nzmax = 0;
    for (const SubDev &s : subs) nzmax = std::max(nzmax, s.nz);
    int zc = zchunk;
    if (zc <= 0 && tail_hidden) {
        // other launches fill this one's last round (tile groups of a batch
        // side by side): whole columns, up to 256 planes per item (64-shot
        // batch, sides 96-256: FP32 346 against 310 Gpts/s with the model
        // below, BF16 343-347 against 339-341)
        zc = (nzmax + (nzmax + 255) / 256 - 1) / ((nzmax + 255) / 256);
    } else if (zc <= 0) {
        // nzc chunks per column, for the lowest modelled step time.  An
        // item costs its planes plus 8 * 0.7 (its z halo is streamed but
        // not computed).  Static schedule: whole rounds of `grid` items.
        // Dynamic: the work spread over `grid` CTAs plus ti.tail item times
        // for the last, uneven round.  At least two chunks per column (one
        // 512-plane item per column: 512^3 1-8 % slower than two), at
        // least 16 planes per item, at most ti.zcap under the dynamic
        // schedule and 512 under the static one (the compensated sum of an
        // item's plane norms then stays within gamma_511^2 = 1e-9).
        // Measured on 512^3 (static): 256-plane items 376 against 353
        // Gpts/s with 64 for FP32.
        const bool dyn = dynamic_schedule(sched, (int)subs.size(), ncols, grid);
        const double halo = 8 * 0.7;
        const int cap = dyn && ti.zcap > 0 ? ti.zcap : 512;
        const int lo = std::max(nzmax >= 32 ? 2 : 1, (nzmax + cap - 1) / cap);
        const int hi = std::max(lo, nzmax / 16);
        double best = 1e300;
        int best_n = lo;
        for (int nzc = lo; nzc <= hi; ++nzc) {
            const double item = (double)nzmax / nzc + halo;
            const long long n = ncols * nzc;
            const double cost = dyn ? (double)n * item / grid + ti.tail * item
                                    : (double)((n + grid - 1) / grid) * item;
            if (cost < best - 1e-9) {
                best = cost;
                best_n = nzc;
            }
        }
        zc = (nzmax + best_n - 1) / best_n;
    }
    struct Key { int z, sub, y, x; };
    std::vector<std::pair<Key, Item>> v;
    for (int si = 0; si < (int)subs.size(); ++si) {
        const SubDev &s = subs[si];
        int nzc = (s.nz + zc - 1) / zc;
        for (int c = 0; c < nzc; ++c) {
            int z0 = (int)((long long)s.nz * c / nzc);
            int z1 = (int)((long long)s.nz * (c + 1) / nzc);
            if (z1 <= z0) continue;
            const int ntx = (s.nx + TX - 1) / TX;
            for (int y0 = 0, row = 0; y0 < s.ny; y0 += TY, ++row)
                for (int x0 = 0, col = 0; x0 < s.nx; x0 += TX, ++col) {
                    Item it{sub_base + si, x0 | (y0 << 16), z0, z1};
                    // within a tile row the columns start at (row mod ntx):
                    // CTA b takes items b, b + grid, ..., and when grid is
                    // a multiple of the row length a plain order would give
                    // each CTA one fixed column -- every partial, edge or
                    // halo-put tile of the grid on the same few CTAs
                    // (1200^3: 5.6 against 4.9 ms per step)
                    const int key = (col + ntx - row % ntx) % ntx;
                    v.push_back({Key{s.gz0 + z0, si, y0, key}, it});
                }
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const auto &a, const auto &b) {
        if (a.first.z != b.first.z) return a.first.z < b.first.z;
        if (a.first.sub != b.first.sub) return a.first.sub < b.first.sub;
        if (a.first.y != b.first.y) return a.first.y < b.first.y;
        return a.first.x < b.first.x;
    });
    items.clear();
    for (auto &p : v) items.push_back(p.second);
    return zc;
}

}  // namespace gw

// ================================================================ C ABI

extern "C" {

gw_status gw_domain_create(gw_ctx *c, const gw_shot_desc *desc, int px, int py,
                           int pz, const int *split_x, const int *split_y,
                           const int *split_z, int symmetric, gw_domain **out)
{
    if (!c || !desc || !out) return fail(GW_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (c->device < 0) return fail(GW_ERR_STATE, "domains need a device context");
    if (!c->base) return fail(GW_ERR_STATE, "no segment attached");
    const gw_shot_desc &D = *desc;
    if (D.nx <= 0 || D.ny <= 0 || D.nz <= 0 || D.h <= 0 || D.nsteps < 0)
        return fail(GW_ERR_ARG, "bad grid %d x %d x %d, h %g", D.nx, D.ny, D.nz, D.h);
    if (D.nx > 65535 || D.ny > 65535)
        return fail(GW_ERR_ARG, "nx, ny must be < 65536");
    if (D.dtype < DT_F32 || D.dtype > DT_BF16) return fail(GW_ERR_ARG, "bad dtype");
    if (D.schedule < GW_SCHED_AUTO || D.schedule > GW_SCHED_DYNAMIC)
        return fail(GW_ERR_ARG, "bad schedule %d", D.schedule);
    for (double sc : {D.scale_u, D.scale_w}) {
        int e2 = 0;
        // the kernels fold the scales into exact power-of-two factors
        if (sc < 0 || (sc > 0 && (std::frexp(sc, &e2) != 0.5 || e2 < -30 || e2 > 30)))
            return fail(GW_ERR_ARG, "scale %g is not a power of two in [2^-31, 2^29]", sc);
    }
    if (px <= 0 || py <= 0 || pz <= 0) return fail(GW_ERR_ARG, "bad decomposition");
    int nsub = px * py * pz;
    if (nsub > c->nranks)
        return fail(GW_ERR_ARG, "%d subdomains need %d ranks; the segment has %d",
                    nsub, nsub, c->nranks);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    GW_TRY_CUDA(cudaSetDevice(c->device));

    gw_domain *d = new (std::nothrow) gw_domain();
    if (!d) return fail(GW_ERR_NOMEM, "out of host memory");
    d->ctx = c;
    d->desc = D;
    if (d->desc.sponge_a <= 0) d->desc.sponge_a = 0.015;
    d->dtype = D.dtype;
    d->delta = D.dtype == DT_F16S || D.dtype == DT_BF16;
    d->np[0] = px; d->np[1] = py; d->np[2] = pz;
    d->symmetric = symmetric != 0;
    d->chunk = D.chunk == 0 ? kDefaultChunk : std::max(1, std::abs(D.chunk));

    auto fail_out = [&](gw_status st) {
        gw_domain_destroy(d);
        return st;
    };

    // ---- decomposition (tensor-product split, rank = (k*py + j)*px + i)
    const int *splits[3] = {split_x, split_y, split_z};
    const int ext[3] = {D.nx, D.ny, D.nz};
    for (int a = 0; a < 3; ++a) {
        int n = ext[a], p = d->np[a];
        d->split[a].assign(p, 0);
        long long sum = 0;
        for (int i = 0; i < p; ++i) {
            int v = splits[a] ? splits[a][i] : n / p + (i < n % p ? 1 : 0);
            if (v <= 0) return fail_out(fail(GW_ERR_ARG, "empty subdomain along axis %d", a));
            if (v < R && (p > 1 || (D.periodic >> a & 1)))
                return fail_out(fail(GW_ERR_ARG, "subdomain thinner than the halo"));
            d->split[a][i] = v;
            sum += v;
        }
        if (sum != n) return fail_out(fail(GW_ERR_ARG, "splits of axis %d do not sum to %d", a, n));
    }
    const int es = dtype_size(d->dtype), xo = dtype_xoff(d->dtype);
    // row pitch: a multiple of 32 bytes (whole sectors, 16-byte TMA strides).
    // A 128-byte multiple left up to 124 bytes of padding per row that the
    // memory system fetched along with the rows (512^3 8 x 1 x 1 x slabs,
    // 64-wide: 96-element rows for 76 used, DRAM reads +41 %; with 80-element
    // rows the step ran 10-13 % faster, and 512^3 undecomposed 1.4 %)
    const int cmul = 32 / es;
    d->subs.assign(nsub, SubDev{});
    int maxn[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
        for (int v : d->split[a]) maxn[a] = std::max(maxn[a], v);
    std::vector<size_t> fbytes(nsub), cbytes(nsub);
    for (int k = 0, gz = 0; k < pz; gz += d->split[2][k], ++k)
        for (int j = 0, gy = 0; j < py; gy += d->split[1][j], ++j)
            for (int i = 0, gx = 0; i < px; gx += d->split[0][i], ++i) {
                int r = (k * py + j) * px + i;
                SubDev &s = d->subs[r];
                s.nx = d->split[0][i]; s.ny = d->split[1][j]; s.nz = d->split[2][k];
                s.gx0 = gx; s.gy0 = gy; s.gz0 = gz;
                // symmetric: every subdomain laid out like the largest one
                int lx = d->symmetric ? maxn[0] : s.nx;
                int ly = d->symmetric ? maxn[1] : s.ny;
                int lz = d->symmetric ? maxn[2] : s.nz;
                s.px = (int)align_up((size_t)(xo + lx + R), (size_t)cmul);
                s.py = ly + 2 * R;
                s.shot = 0;
                s.rank = r;
                size_t elems = (size_t)s.px * s.py * (size_t)(lz + 2 * R);
                fbytes[r] = elems * es;
                cbytes[r] = elems * (d->delta ? 2 : es);
                int ii[3] = {i, j, k};
                for (int a = 0; a < 3; ++a)
                    for (int side = 0; side < 2; ++side) {
                        int q[3] = {ii[0], ii[1], ii[2]};
                        q[a] += side ? 1 : -1;
                        bool wrap = (D.periodic >> a) & 1;
                        if (q[a] < 0 || q[a] >= d->np[a]) {
                            if (!wrap) { s.nbr[2 * a + side] = -1; continue; }
                            q[a] = (q[a] + d->np[a]) % d->np[a];
                        }
                        s.nbr[2 * a + side] = (q[2] * py + q[1]) * px + q[0];
                    }
            }

    // ---- PGAS allocation of the fields
    const int nf = d->delta ? 4 : 3;
    const int fields[4] = {0, 1, 3, 2};   // u0, u1, coef, (w)
    for (int fi = 0; fi < nf; ++fi) {
        int f = fields[fi];
        gw_gptr g = 0;
        gw_status st;
        if (d->symmetric) {
            size_t b = f == 3 ? cbytes[0] : fbytes[0];
            st = ctx_alloc_sym(c, b, &g);
            if (st == GW_OK) d->device_bytes += align_up(b, kAlign) * nsub;
        } else {
            std::vector<size_t> b(c->nranks, 0);
            for (int r = 0; r < nsub; ++r) b[r] = f == 3 ? cbytes[r] : fbytes[r];
            st = ctx_alloc_asym(c, b.data(), &g);
            if (st == GW_OK)
                for (int r = 0; r < nsub; ++r) d->device_bytes += align_up(b[r], kAlign);
        }
        if (st != GW_OK) return fail_out(st);
        d->allocs.push_back(g);
        d->g_fields[f] = g;
        for (int r = 0; r < nsub; ++r) {
            char *p = nullptr;
            size_t sz = 0;
            // asymmetric: a second-level pointer fetch, then the cache
            gw_status rs = ctx_resolve(c, g, r, &p, &sz);
            if (rs != GW_OK) return fail_out(rs);
            cudaError_t e = cudaMemset(p, 0, sz);
            if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaMemset"));
            SubDev &s = d->subs[r];
            if (f == 0) s.u[0] = p;
            else if (f == 1) s.u[1] = p;
            else if (f == 2) s.w = p;
            else s.coef = p;
        }
    }

    // ---- metadata
    const int cap = std::max(1, D.nsteps);
    size_t off_subs = 0;
    size_t off_shot = align_up(off_subs + sizeof(SubDev) * nsub, kAlign);
    size_t off_maps = align_up(off_shot + sizeof(ShotDev), kAlign);
    size_t off_err = align_up(off_maps + 128 * kMapsPerSub * (size_t)nsub, kAlign);
    size_t off_step = off_err + 64;
    size_t off_scr = off_err + 128;
    size_t off_wl = align_up(off_scr + 64, kAlign);
    size_t off_norm = align_up(off_wl + sizeof(double) * kMaxSources * (size_t)cap, kAlign);
    size_t off_g = align_up(off_norm + sizeof(double) * (size_t)cap, kAlign);
    size_t off_src = align_up(off_g + sizeof(double) * (size_t)(D.nx + D.ny + D.nz), kAlign);
    size_t off_halo = align_up(off_src + sizeof(int4) * kMaxSources, kAlign);
    size_t off_chk = align_up(off_halo + sizeof(HaloDesc) * 6 * (size_t)nsub, kAlign);
    size_t planes = 0;
    for (const SubDev &s : d->subs) planes += (size_t)s.nz;
    size_t total = align_up(off_chk + 3 * sizeof(double) * planes, kAlign);
    char *m = nullptr;
    gw_status st = local_alloc(d, total, &m);
    if (st != GW_OK) return fail_out(st);
    cudaError_t e = cudaMemset(m, 0, total);
    if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaMemset"));
    d->d_subs = reinterpret_cast<SubDev *>(m + off_subs);
    d->d_shot = reinterpret_cast<ShotDev *>(m + off_shot);
    d->d_maps = m + off_maps;
    d->d_err = reinterpret_cast<unsigned *>(m + off_err);
    d->d_step = reinterpret_cast<int *>(m + off_step);
    d->d_gbar = reinterpret_cast<unsigned *>(m + off_err + 32);
    d->d_ctr = reinterpret_cast<unsigned *>(m + off_err + 96);
    d->d_scratch = reinterpret_cast<double *>(m + off_scr);
    d->d_wavelet = reinterpret_cast<double *>(m + off_wl);
    d->d_norms = reinterpret_cast<double *>(m + off_norm);
    d->d_gtab = reinterpret_cast<double *>(m + off_g);
    d->d_src = reinterpret_cast<int4 *>(m + off_src);
    d->d_halo = reinterpret_cast<HaloDesc *>(m + off_halo);
    d->d_chk = reinterpret_cast<double *>(m + off_chk);

    // sponge tables on global coordinates, FP64 (the kernels round them to
    // their arithmetic type when they load them)
    {
        std::vector<double> g(D.nx + D.ny + D.nz);
        const int n3[3] = {D.nx, D.ny, D.nz};
        size_t o = 0;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < n3[a]; ++i)
                g[o++] = cerjan(i, n3[a], D.sponge, d->desc.sponge_a);
        e = cudaMemcpy(d->d_gtab, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaMemcpy"));
    }
    ShotDev &sh = d->shot;
    sh.step = d->d_step;
    sh.wavelet = d->d_wavelet;
    sh.traces = nullptr;
    sh.norms = d->d_norms;
    sh.gx = d->d_gtab;
    sh.gy = d->d_gtab + D.nx;
    sh.gz = d->d_gtab + D.nx + D.ny;
    sh.src = d->d_src;
    sh.rec = nullptr;
    sh.cap = cap;
    sh.limit = INT_MAX;
    sh.nsrc = 0;
    sh.nrec = 0;
    sh.NX = D.nx; sh.NY = D.ny; sh.NZ = D.nz;
    sh.su = sh.sw = sh.isu = sh.isw = 1.0f;

    e = cudaMemcpy(d->d_subs, d->subs.data(), sizeof(SubDev) * nsub, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaMemcpy"));
    build_halo_plan(d);
    if (!d->halo.empty()) {
        e = cudaMemcpy(d->d_halo, d->halo.data(), sizeof(HaloDesc) * d->halo.size(),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaMemcpy"));
    }
    st = plan_schedule(d);
    if (st != GW_OK) return fail_out(st);
    st = make_maps(d);
    if (st != GW_OK) return fail_out(st);
    st = push_shot(d);
    if (st != GW_OK) return fail_out(st);
    *out = d;
    return GW_OK;
}

gw_status gw_domain_destroy(gw_domain *d)
{
    if (!d) return GW_OK;
    gw_ctx *c = d->ctx;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->device >= 0) {
        cudaSetDevice(c->device);
        cudaDeviceSynchronize();
    }
    destroy_graph(d);
    if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
    harvest_events(d);
    for (cudaEvent_t e : d->ev_pool) cudaEventDestroy(e);
    for (gw_gptr g : d->allocs) ctx_free(c, g);
    delete d;
    return GW_OK;
}

gw_status gw_domain_info_get(gw_domain *d, gw_domain_info *out)
{
    if (!d || !out) return fail(GW_ERR_ARG, "NULL argument");
    out->dt = d->dt;
    out->courant = d->courant;
    out->vmax = d->vmax;
    out->nsub = d->nsub();
    out->step = d->step;
    out->tile = d->cfg + 1;
    out->ctas = d->grid;
    out->items = d->nitems;
    out->scale_u = d->su;
    out->scale_w = d->sw;
    out->device_bytes = d->device_bytes;
    out->schedule = d->dynamic ? GW_SCHED_DYNAMIC : GW_SCHED_STATIC;
    return GW_OK;
}

static void choose_scales(gw_domain *d);

// dt from the model's largest velocity (fixed dt, Courant number, or half
// the stability limit), and the Courant number that results.
static void set_time_step(gw_domain *d, double vmax)
{
    const gw_shot_desc &D = d->desc;
    d->vmax = vmax;
    if (D.dt > 0) {
        d->dt = D.dt;
    } else {
        double nu = D.courant > 0 ? D.courant : 0.5 * nu_limit();
        d->dt = nu * D.h / vmax;
    }
    d->courant = vmax * d->dt / D.h;
}

static gw_status set_model_impl(gw_domain *d, const void *vel, bool f32)
{
    GW_TRY(check_dom(d));
    if (!vel) return fail(GW_ERR_ARG, "vel is NULL");
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    const gw_shot_desc &D = d->desc;
    const size_t vs = f32 ? 4 : 8;
    const size_t plane = (size_t)D.nx * D.ny;
    Stage st;
    GW_TRY(stage_alloc(d, st, plane * D.nz * vs + 16, plane * vs));
    unsigned long long *d_max = reinterpret_cast<unsigned long long *>(d->d_scratch);
    GW_TRY_CUDA(cudaMemset(d_max, 0, sizeof *d_max));
    const char *h = static_cast<const char *>(vel);
    // When the coef array holds the input velocities exactly (FP32 coef and
    // FP32 input, or FP64 coef), the model crosses to the device once: the
    // first pass stores v in the coef array while it finds vmax, and coef =
    // (v dt / h)^2 is then formed in place -- the same FP64 product of the
    // same v, so the same bits as from the host copy.  Otherwise a second
    // pass reads the host model again.
    const bool once = d->dtype == DT_F64 || (d->dtype == DT_F32 && f32);
    // pass 1: vmax on the GPU
    GW_TRY(upload_slabs(d, st, h, plane * vs, [&](char *buf, int z, int zh) -> gw_status {
        GW_TRY_CUDA(launch_vmax(buf, plane * (size_t)(zh - z), f32, d_max, nullptr));
        if (once) {
            ModelSlab ms{buf, f32 ? 1 : 0, D.nx, D.ny, z, zh, 0.0, 0, 1};
            for (const SubDev &s : d->subs)
                GW_TRY_CUDA(launch_coef(ms, s, d->dtype, nullptr));
        }
        return GW_OK;
    }));
    unsigned long long bits = 0;
    GW_TRY_CUDA(cudaMemcpy(&bits, d_max, sizeof bits, cudaMemcpyDeviceToHost));
    double vmax;
    std::memcpy(&vmax, &bits, sizeof vmax);
    if (!(vmax > 0) || !std::isfinite(vmax))
        return fail(GW_ERR_ARG, "velocity model must be positive and finite");
    set_time_step(d, vmax);
    if (once) {
        for (const SubDev &s : d->subs)
            GW_TRY_CUDA(launch_coef_square(s, d->dtype, d->dt / D.h, nullptr));
    } else {
        // pass 2: coef = (v dt / h)^2 in FP64 on the GPU, rounded to storage
        GW_TRY(upload_slabs(d, st, h, plane * vs, [&](char *buf, int z, int zh) -> gw_status {
            ModelSlab ms{buf, f32 ? 1 : 0, D.nx, D.ny, z, zh, d->dt / D.h, 0, 0};
            for (const SubDev &s : d->subs)
                GW_TRY_CUDA(launch_coef(ms, s, d->dtype, nullptr));
            return GW_OK;
        }));
    }
    // the legacy stream only: work of other shots on other streams runs on
    GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    d->model_set = true;
    choose_scales(d);
    return push_shot(d);
}

gw_status gw_set_model_layered(gw_domain *d, const double *vz)
{
    GW_TRY(check_dom(d));
    if (!vz) return fail(GW_ERR_ARG, "vz is NULL");
    const gw_shot_desc &D = d->desc;
    double vmax = 0;
    for (int z = 0; z < D.nz; ++z) {
        if (!(vz[z] > 0) || !std::isfinite(vz[z]))
            return fail(GW_ERR_ARG, "velocity model must be positive and finite");
        vmax = std::max(vmax, vz[z]);
    }
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    Stage st;
    GW_TRY(stage_alloc(d, st, sizeof(double) * D.nz + 16, sizeof(double) * D.nz));
    set_time_step(d, vmax);
    GW_TRY_CUDA(cudaMemcpy(st.p, vz, sizeof(double) * D.nz, cudaMemcpyHostToDevice));
    ModelSlab ms{st.p, 0, D.nx, D.ny, 0, D.nz, d->dt / D.h, 1};
    for (const SubDev &s : d->subs)
        GW_TRY_CUDA(launch_coef(ms, s, d->dtype, nullptr));
    GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    d->model_set = true;
    choose_scales(d);
    return push_shot(d);
}

gw_status gw_set_model(gw_domain *d, const double *vel) { return set_model_impl(d, vel, false); }
gw_status gw_set_model_f32(gw_domain *d, const float *vel) { return set_model_impl(d, vel, true); }

gw_status gw_ricker(double f, double dt, int n, float *out)
{
    if (f <= 0 || dt <= 0 || n < 0 || (n && !out)) return fail(GW_ERR_ARG, "bad Ricker arguments");
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double tau = i * dt - 1.0 / f;
        double a = pi * pi * f * f * tau * tau;
        out[i] = (float)((1.0 - 2.0 * a) * std::exp(-a));
    }
    return GW_OK;
}

gw_status gw_round_to_f32(const double *in_dev, float *out_dev, size_t n, gw_stream stream)
{
    if (n && (!in_dev || !out_dev)) return fail(GW_ERR_ARG, "NULL array");
    GW_TRY_CUDA(launch_round_to_f32(in_dev, out_dev, n, static_cast<cudaStream_t>(stream)));
    return GW_OK;
}

// Power-of-two scales of FP16 delta storage: keep the largest expected
// |u| near 2^12 (16x headroom below the FP16 maximum) and w four times
// larger (w ~ u * omega * dt is smaller than u).
static void choose_scales(gw_domain *d)
{
    if (d->dtype != DT_F16S) {
        d->su = d->sw = 1.0;
    } else {
        double amp = 0.0;
        const double cmax = d->courant * d->courant;
        for (const std::vector<double> &w : d->wavelets) {
            // sum of |wavelet| bounds the accumulated kick at the source
            double acc = 0.0;
            for (double v : w) acc += std::fabs(v);
            amp += cmax * acc;
        }
        if (amp <= 0) amp = 1.0;
        double k = std::floor(std::log2(4096.0 / amp));
        k = std::max(-20.0, std::min(20.0, k));
        d->su = std::ldexp(1.0, (int)k);
        d->sw = d->su * 4.0;
        if (d->desc.scale_u > 0) d->su = d->desc.scale_u;
        if (d->desc.scale_w > 0) d->sw = d->desc.scale_w;
    }
    d->shot.su = (float)d->su;
    d->shot.sw = (float)d->sw;
    d->shot.isu = (float)(1.0 / d->su);
    d->shot.isw = (float)(1.0 / d->sw);
}

static gw_status add_source(gw_domain *d, int gx, int gy, int gz,
                            std::vector<double> w)
{
    GW_TRY(check_dom(d));
    const gw_shot_desc &D = d->desc;
    if (gx < 0 || gy < 0 || gz < 0 || gx >= D.nx || gy >= D.ny || gz >= D.nz)
        return fail(GW_ERR_ARG, "source (%d, %d, %d) outside the grid", gx, gy, gz);
    if ((int)d->srcs.size() >= kMaxSources) return fail(GW_ERR_ARG, "too many sources");
    if (d->step != 0 && d->dtype == DT_F16S)
        return fail(GW_ERR_STATE, "FP16 scales are fixed once stepping started");
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    int idx = (int)d->srcs.size();
    w.resize(d->shot.cap, 0.0);
    GW_TRY_CUDA(cudaMemcpy(d->d_wavelet + (size_t)idx * d->shot.cap, w.data(),
                           sizeof(double) * w.size(), cudaMemcpyHostToDevice));
    d->srcs.push_back(make_int4(gx, gy, gz, 0));
    d->wavelets.push_back(std::move(w));
    GW_TRY_CUDA(cudaMemcpy(d->d_src, d->srcs.data(), sizeof(int4) * d->srcs.size(),
                           cudaMemcpyHostToDevice));
    d->shot.nsrc = (int)d->srcs.size();
    choose_scales(d);
    return push_shot(d);
}

gw_status gw_inject_source(gw_domain *d, int gx, int gy, int gz,
                           const float *wavelet, int n)
{
    if (!d) return fail(GW_ERR_ARG, "domain is NULL");
    if (n < 0 || (n && !wavelet)) return fail(GW_ERR_ARG, "bad wavelet");
    std::vector<double> w(wavelet, wavelet + n);
    return add_source(d, gx, gy, gz, std::move(w));
}

gw_status gw_inject_ricker(gw_domain *d, int gx, int gy, int gz, double f_peak)
{
    if (!d) return fail(GW_ERR_ARG, "domain is NULL");
    if (!d->model_set) return fail(GW_ERR_STATE, "set the velocity model first (dt)");
    if (!(f_peak > 0)) return fail(GW_ERR_ARG, "peak frequency must be positive");
    std::vector<double> w(d->shot.cap);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < d->shot.cap; ++i) {
        double tau = i * d->dt - 1.0 / f_peak;
        double a = pi * pi * f_peak * f_peak * tau * tau;
        w[i] = (1.0 - 2.0 * a) * std::exp(-a);
    }
    return add_source(d, gx, gy, gz, std::move(w));
}

// Most sources + receivers inside any one work item of the domain (the
// kernel keeps at most kMaxLocal per item).
static int most_per_item(const gw_domain *d, const std::vector<int4> &recs)
{
    int most = 0;
    for (const Item &it : d->items) {
        const SubDev &s = d->subs[it.sub];
        const int x0 = s.gx0 + (it.xy & 0xffff), y0 = s.gy0 + (it.xy >> 16);
        const int x1 = std::min(x0 + d->ti.tx, s.gx0 + s.nx), y1 = std::min(y0 + d->ti.ty, s.gy0 + s.ny);
        const int z0 = s.gz0 + it.z0, z1 = s.gz0 + it.z1;
        int n = 0;
        for (const std::vector<int4> *l : {&d->srcs, &recs})
            for (const int4 &q : *l)
                n += q.x >= x0 && q.x < x1 && q.y >= y0 && q.y < y1 && q.z >= z0 && q.z < z1;
        most = std::max(most, n);
    }
    return most;
}

gw_status gw_set_receivers(gw_domain *d, int nrec, const int *xyz)
{
    GW_TRY(check_dom(d));
    if (nrec < 0 || (nrec && !xyz)) return fail(GW_ERR_ARG, "bad receivers");
    const gw_shot_desc &D = d->desc;
    std::vector<int4> r(nrec);
    for (int i = 0; i < nrec; ++i) {
        int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (x < 0 || y < 0 || z < 0 || x >= D.nx || y >= D.ny || z >= D.nz)
            return fail(GW_ERR_ARG, "receiver %d outside the grid", i);
        r[i] = make_int4(x, y, z, 0);
    }
    if (nrec > kMaxLocal - (int)d->srcs.size()) {
        const int most = most_per_item(d, r);
        if (most > kMaxLocal)
            return fail(GW_ERR_ARG, "%d sources and receivers fall in one work item (at most %d); "
                        "spread them or use a smaller zchunk", most, kMaxLocal);
    }
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    if (d->g_rec) { drop_alloc(d, d->g_rec); d->g_rec = 0; d->d_rec = nullptr; }
    if (d->g_traces) { drop_alloc(d, d->g_traces); d->g_traces = 0; d->d_traces = nullptr; }
    if (nrec) {
        char *p = nullptr;
        GW_TRY(local_alloc(d, sizeof(int4) * nrec, &p, &d->g_rec));
        d->d_rec = reinterpret_cast<int4 *>(p);
        GW_TRY_CUDA(cudaMemcpy(d->d_rec, r.data(), sizeof(int4) * nrec, cudaMemcpyHostToDevice));
        size_t tb = sizeof(float) * (size_t)nrec * d->shot.cap;
        GW_TRY(local_alloc(d, tb, &p, &d->g_traces));
        d->d_traces = reinterpret_cast<float *>(p);
        GW_TRY_CUDA(cudaMemset(d->d_traces, 0, tb));
    }
    d->nrec = nrec;
    d->recs = r;
    d->shot.nrec = nrec;
    d->shot.rec = d->d_rec;
    d->shot.traces = d->d_traces;
    return push_shot(d);
}

gw_status gw_step(gw_domain *d, int nsteps, gw_stream stream)
{
    GW_TRY(check_dom(d));
    if (nsteps < 0) return fail(GW_ERR_ARG, "negative step count");
    if (!d->model_set) return fail(GW_ERR_STATE, "set the velocity model first");
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    d->last = s;
    int left = nsteps;
    const bool graphs = d->desc.chunk >= 0 && !d->timing;
    while (left > 0) {
        if (graphs && left >= d->chunk) {
            GW_TRY(ensure_graph(d));
            GW_TRY_CUDA(cudaGraphLaunch(d->gexec, s));
            left -= d->chunk;
            d->step = std::min(d->step + d->chunk, d->shot.limit);
        } else {
            int nk = std::min(left, d->chunk);
            GW_TRY(enqueue_chunk(d, nk, s, d->timing));
            left -= nk;
            d->step = std::min(d->step + nk, d->shot.limit);
        }
    }
    return GW_OK;
}

gw_status gw_put_halo(gw_domain *d, gw_stream stream)
{
    GW_TRY(check_dom(d));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    if (d->halo.empty()) return GW_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    d->last = s;
    GW_TRY_CUDA(launch_halo(d->d_halo, (int)d->halo.size(), d->halo_units, d->d_subs,
                            d->d_step, -1, d->dtype, s));
    return GW_OK;
}

gw_status gw_barrier(gw_domain *d, gw_stream stream, int sync)
{
    GW_TRY(check_dom(d));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // puts issued on another stream become visible to `s` from here on
    if (d->last && d->last != s) {
        cudaEvent_t ev;
        GW_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, d->last);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return cuda_fail(e, "barrier join");
    }
    GW_TRY(gw_fence(d->ctx, stream));
    if (sync) {
        GW_TRY_CUDA(cudaStreamSynchronize(s));
        return sync_dom(d);
    }
    return GW_OK;
}

gw_status gw_read_receivers(gw_domain *d, float *out, int nrec, int nsteps)
{
    GW_TRY(check_dom(d));
    if (nrec < 0 || nrec > d->nrec || nsteps < 0 || nsteps > d->shot.cap || (!out && nrec && nsteps))
        return fail(GW_ERR_ARG, "bad receiver read (%d of %d receivers, %d steps)", nrec,
                    d->nrec, nsteps);
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    if (nrec && nsteps)
        GW_TRY_CUDA(cudaMemcpy2D(out, sizeof(float) * nsteps, d->d_traces,
                                 sizeof(float) * d->shot.cap, sizeof(float) * nsteps, nrec,
                                 cudaMemcpyDeviceToHost));
    return GW_OK;
}

static gw_status field_index(gw_domain *d, int which, int *f, double *scale)
{
    *scale = 1.0;
    switch (which) {
    case GW_FIELD_U: *f = 0; *scale = d->su; return GW_OK;
    case GW_FIELD_UPREV: *f = 1; *scale = d->su; return GW_OK;
    case GW_FIELD_W:
        if (!d->delta) return fail(GW_ERR_ARG, "GW_FIELD_W needs delta (16-bit) storage");
        *f = 2; *scale = d->sw; return GW_OK;
    case GW_FIELD_COEF: *f = 3; return GW_OK;
    default: return fail(GW_ERR_ARG, "unknown field %d", which);
    }
}

gw_status gw_read_wavefield(gw_domain *d, int which, void *out, int f64)
{
    GW_TRY(check_dom(d));
    if (!out) return fail(GW_ERR_ARG, "out is NULL");
    int f = 0;
    double scale;
    GW_TRY(field_index(d, which, &f, &scale));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    const gw_shot_desc &D = d->desc;
    const size_t es = f64 ? 8 : 4, plane = (size_t)D.nx * D.ny;
    Stage st;
    GW_TRY(stage_alloc(d, st, plane * D.nz * es, plane * es));
    int pps = planes_per_slab(d, es, st.bytes);
    char *h = static_cast<char *>(out);
    for (int z = 0; z < D.nz; z += pps) {
        int zh = std::min(D.nz, z + pps);
        FieldSlab fs{st.p, f64, D.nx, D.ny, z, zh, f, d->step & 1, scale};
        for (const SubDev &s : d->subs) GW_TRY_CUDA(launch_gather(fs, s, d->dtype, nullptr));
        GW_TRY_CUDA(cudaMemcpy(h + plane * (size_t)z * es, st.p, plane * (size_t)(zh - z) * es,
                               cudaMemcpyDeviceToHost));
    }
    return GW_OK;
}

gw_status gw_write_wavefield(gw_domain *d, int which, const void *in, int f64)
{
    GW_TRY(check_dom(d));
    if (!in) return fail(GW_ERR_ARG, "input is NULL");
    if (which == GW_FIELD_UPREV && d->delta)
        return fail(GW_ERR_ARG, "delta storage: write GW_FIELD_W (w = u_n - G u_{n-1})");
    if (which == GW_FIELD_COEF) return fail(GW_ERR_ARG, "set coef through gw_set_model");
    int f = 0;
    double scale;
    GW_TRY(field_index(d, which, &f, &scale));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    const gw_shot_desc &D = d->desc;
    const size_t es = f64 ? 8 : 4, plane = (size_t)D.nx * D.ny;
    Stage st;
    GW_TRY(stage_alloc(d, st, plane * D.nz * es, plane * es));
    int pps = planes_per_slab(d, es, st.bytes);
    const char *h = static_cast<const char *>(in);
    for (int z = 0; z < D.nz; z += pps) {
        int zh = std::min(D.nz, z + pps);
        GW_TRY_CUDA(cudaMemcpy(st.p, h + plane * (size_t)z * es, plane * (size_t)(zh - z) * es,
                               cudaMemcpyHostToDevice));
        FieldSlab fs{st.p, f64, D.nx, D.ny, z, zh, f, d->step & 1, scale};
        for (const SubDev &s : d->subs) GW_TRY_CUDA(launch_scatter(fs, s, d->dtype, nullptr));
    }
    // refresh the face halos of the written field
    if (!d->halo.empty() && (f == 0 || f == 1))
        GW_TRY_CUDA(launch_halo(d->d_halo, (int)d->halo.size(), d->halo_units, d->d_subs,
                                d->d_step, f == 0 ? -1 : -2, d->dtype, nullptr));
    GW_TRY_CUDA(cudaDeviceSynchronize());
    return GW_OK;
}

gw_status gw_norms(gw_domain *d, double *out, int n)
{
    GW_TRY(check_dom(d));
    if (n < 0 || n > d->step || n > d->shot.cap || (n && !out))
        return fail(GW_ERR_ARG, "bad norm read (%d of %d steps)", n, d->step);
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    if (n) GW_TRY_CUDA(cudaMemcpy(out, d->d_norms, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return GW_OK;
}

gw_status gw_check(gw_domain *d, double *norm2, double *energy)
{
    GW_TRY(check_dom(d));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    int planes = 0;
    for (const SubDev &s : d->subs) {
        GW_TRY_CUDA(launch_check(s, d->step & 1, d->dtype, d->su, d->d_chk + 3 * planes,
                                 nullptr));
        planes += s.nz;
    }
    GW_TRY_CUDA(launch_check_sum(d->d_chk, planes, d->d_scratch, nullptr));
    double a[3];
    GW_TRY_CUDA(cudaMemcpy(a, d->d_scratch, sizeof a, cudaMemcpyDeviceToHost));
    if (norm2) *norm2 = a[0];
    if (energy) *energy = a[1] - a[2];
    if (!std::isfinite(a[0]) || !std::isfinite(a[1]) || !std::isfinite(a[2]))
        return fail(GW_ERR_NUMERIC, "non-finite check reduction");
    return GW_OK;
}

gw_status gw_kernel_timing(gw_domain *d, int enable)
{
    GW_TRY(check_dom(d));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    d->timing = enable != 0;
    return GW_OK;
}

gw_status gw_kernel_stats_get(gw_domain *d, gw_kernel_stats *out)
{
    GW_TRY(check_dom(d));
    if (!out) return fail(GW_ERR_ARG, "out is NULL");
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    harvest_events(d);
    out->launches = d->acc_n;
    out->total_ms = d->acc_ms;
    out->halo_ms = d->acc_halo_ms;
    d->acc_n = 0;
    d->acc_ms = d->acc_halo_ms = 0;
    return GW_OK;
}

gw_status gw_state_bytes(gw_domain *d, size_t *bytes)
{
    if (!d || !bytes) return fail(GW_ERR_ARG, "NULL argument");
    size_t b = 16;
    const int nf = d->delta ? 3 : 2;
    for (const SubDev &s : d->subs) {
        size_t el = (size_t)s.px * s.py * (size_t)(s.nz + 2 * R);
        b += (size_t)nf * el * d->esize();
    }
    *bytes = b;
    return GW_OK;
}

static gw_status state_copy(gw_domain *d, char *host, bool save)
{
    GW_TRY(check_dom(d));
    std::lock_guard<std::recursive_mutex> lk(d->ctx->mu);
    GW_TRY(sync_dom(d));
    int hdr[4] = {d->step, d->nsub(), d->dtype, 0};
    if (save) {
        std::memcpy(host, hdr, sizeof hdr);
    } else {
        int got[4];
        std::memcpy(got, host, sizeof got);
        if (got[1] != d->nsub() || got[2] != d->dtype)
            return fail(GW_ERR_ARG, "state does not match this domain");
        d->step = got[0];
        GW_TRY_CUDA(cudaMemcpy(d->d_step, &d->step, sizeof(int), cudaMemcpyHostToDevice));
    }
    size_t off = 16;
    const int nf = d->delta ? 3 : 2;
    for (const SubDev &s : d->subs) {
        size_t el = (size_t)s.px * s.py * (size_t)(s.nz + 2 * R) * d->esize();
        char *f[3] = {s.u[0], s.u[1], s.w};
        for (int i = 0; i < nf; ++i) {
            if (save)
                GW_TRY_CUDA(cudaMemcpy(host + off, f[i], el, cudaMemcpyDeviceToHost));
            else
                GW_TRY_CUDA(cudaMemcpy(f[i], host + off, el, cudaMemcpyHostToDevice));
            off += el;
        }
    }
    return GW_OK;
}

gw_status gw_save_state(gw_domain *d, void *out)
{
    if (!out) return fail(GW_ERR_ARG, "out is NULL");
    return state_copy(d, static_cast<char *>(out), true);
}

gw_status gw_load_state(gw_domain *d, const void *in)
{
    if (!in) return fail(GW_ERR_ARG, "input is NULL");
    return state_copy(d, const_cast<char *>(static_cast<const char *>(in)), false);
}

}  // extern "C"

extern "C" gw_status gw_domain_bytes(const gw_shot_desc *desc, int px, int py, int pz,
                                     int nrec, size_t *out)
{
    if (!desc || !out || px <= 0 || py <= 0 || pz <= 0 || nrec < 0)
        return fail(GW_ERR_ARG, "bad arguments");
    const gw_shot_desc &D = *desc;
    if (D.nx <= 0 || D.ny <= 0 || D.nz <= 0 || D.dtype < DT_F32 || D.dtype > DT_BF16)
        return fail(GW_ERR_ARG, "bad grid or storage type");
    const bool delta = D.dtype == DT_F16S || D.dtype == DT_BF16;
    const int es = dtype_size(D.dtype), xo = dtype_xoff(D.dtype);
    const size_t nsub = (size_t)px * py * pz;
    // symmetric layout: every subdomain padded like the largest one
    const int lx = (D.nx + px - 1) / px, ly = (D.ny + py - 1) / py, lz = (D.nz + pz - 1) / pz;
    const size_t pitch = align_up((size_t)(xo + lx + R), (size_t)(32 / es));
    const size_t elems = pitch * (size_t)(ly + 2 * R) * (size_t)(lz + 2 * R);
    // u0, u1 (and w in the delta form) in the storage type, coef in FP16
    // for the 16-bit types
    size_t total = (delta ? 3 : 2) * align_up(elems * es, kAlign) * nsub;
    total += align_up(elems * (delta ? 2 : es), kAlign) * nsub;
    // metadata, tensor maps, tables (as laid out by gw_domain_create)
    const size_t cap = (size_t)std::max(1, D.nsteps);
    total += align_up(sizeof(SubDev) * nsub, kAlign) + 2 * kAlign +
             align_up(128 * kMapsPerSub * nsub, kAlign) + kAlign +
             align_up(sizeof(double) * kMaxSources * cap, kAlign) +
             align_up(sizeof(double) * cap, kAlign) +
             align_up(sizeof(double) * (size_t)(D.nx + D.ny + D.nz), kAlign) +
             align_up(sizeof(int4) * kMaxSources, kAlign) +
             align_up(sizeof(HaloDesc) * 6 * nsub, kAlign) +
             align_up(3 * sizeof(double) * (size_t)lz * nsub, kAlign);
    // work items and one chunk of norm partials, bounded with the smallest
    // tile extents (32 x 7) and items of at least 32 planes
    const size_t chunk = D.chunk == 0 ? kDefaultChunk : (size_t)std::max(1, std::abs(D.chunk));
    const size_t items = nsub * (size_t)((lx + 31) / 32) * (size_t)((ly + 6) / 7) *
                         (size_t)std::max(1, lz / 32);
    total += align_up((sizeof(Item) + sizeof(double) * chunk) * items + kAlign, kAlign);
    // receivers and their traces
    if (nrec)
        total += align_up(sizeof(int4) * nrec, kAlign) +
                 align_up(sizeof(float) * (size_t)nrec * cap, kAlign);
    *out = total;
    return GW_OK;
}
