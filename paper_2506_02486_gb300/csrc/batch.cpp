// batch.cpp -- several independent shots advanced by the same launches
// (one launch per step, or per chunk of steps in persistent mode, covering
// the work items of every shot), and the kernel-tile autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "domain_impl.h"

using namespace gw;

namespace {

// Shots that can share one launch: same kernel tile, sponge variant and
// neighbour-address mode.
struct Group {
    int cfg = 0;
    bool sponge = false;
    bool symmetric = true;
    bool separate = false;      // halos copied by a kernel after each step
    TileInfo ti{};
    std::vector<gw_domain *> doms;
    std::vector<SubDev> subs;
    std::vector<ShotDev> shots;
    std::vector<Item> items;
    gw_gptr g_meta = 0;
    SubDev *d_subs = nullptr;
    ShotDev *d_shots = nullptr;
    Item *d_items = nullptr;
    char *d_maps = nullptr;
    double *d_partials = nullptr;
    unsigned *d_gbar = nullptr;
    unsigned *d_ctr = nullptr;      // work-item tickets
    bool dynamic = true;            // dynamic schedule unless every shot asks for static
    unsigned *err = nullptr;    // the first shot's device error word
    int grid = 0;
};

}  // namespace

struct gw_batch {
    gw_ctx *ctx = nullptr;
    int dtype = 0;
    int chunk = kDefaultChunk;
    bool graphs = true;
    bool persistent = false;
    std::vector<Group> groups;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;          // one chunk of every group
    // groups launched side by side within a chunk (non-persistent batches
    // of more than one group): streams forked from the caller's and joined
    // at the end of the chunk
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<int> ev_steps;
    double acc_ms = 0;
    int acc_n = 0;
};

namespace {

gw_status build_group(gw_batch *b, Group &g)
{
    gw_ctx *c = b->ctx;
    long long pts = 0;
    for (gw_domain *d : g.doms)
        pts += (long long)d->desc.nx * d->desc.ny * d->desc.nz;
    int occ = step_cfg_occupancy(b->dtype, g.cfg, g.sponge);
    if (occ <= 0) return fail(GW_ERR_CUDA, "kernel configuration does not fit an SM");
    const int G = std::max(1, c->num_sms * occ);
    // concatenate subdomains, shots and work items; each shot's items stay
    // contiguous so that the norm reduction can run per shot
    for (size_t si = 0; si < g.doms.size(); ++si) {
        gw_domain *d = g.doms[si];
        const int base = (int)g.subs.size();
        for (SubDev s : d->subs) {
            s.shot = (int)si;
            for (int f = 0; f < 6; ++f)
                if (s.nbr[f] >= 0) s.nbr[f] += base;
            g.subs.push_back(s);
        }
        long long dp = (long long)d->desc.nx * d->desc.ny * d->desc.nz;
        int share = (int)std::max<long long>(1, (long long)G * dp / std::max(1LL, pts));
        std::vector<Item> it;
        make_items(d->subs, g.ti, share, d->desc.zchunk,
                   g.dynamic ? GW_SCHED_DYNAMIC : GW_SCHED_STATIC, it, base,
                   !b->persistent && b->groups.size() > 1);
        ShotDev sh = d->shot;
        sh.first_item = (int)g.items.size();
        sh.nitems = (int)it.size();
        g.shots.push_back(sh);
        g.items.insert(g.items.end(), it.begin(), it.end());
    }
    const int nsub = (int)g.subs.size(), nsh = (int)g.shots.size();
    const int nit = (int)g.items.size();
    if (nit == 0) return fail(GW_ERR_ARG, "batch has no work");
    g.grid = std::min(G, nit);
    const size_t o_subs = 0;
    const size_t o_shots = align_up(o_subs + sizeof(SubDev) * nsub, kAlign);
    const size_t o_items = align_up(o_shots + sizeof(ShotDev) * nsh, kAlign);
    const size_t o_maps = align_up(o_items + sizeof(Item) * nit, kAlign);
    const size_t o_part = align_up(o_maps + 128 * kMapsPerSub * (size_t)nsub, kAlign);
    const size_t o_bar = align_up(o_part + sizeof(double) * nit * (size_t)std::max(1, b->chunk), kAlign);
    const size_t total = o_bar + kAlign;
    char *m = nullptr;
    GW_TRY(ctx_alloc_local(c, 0, total, &g.g_meta, &m));
    g.d_subs = reinterpret_cast<SubDev *>(m + o_subs);
    g.d_shots = reinterpret_cast<ShotDev *>(m + o_shots);
    g.d_items = reinterpret_cast<Item *>(m + o_items);
    g.d_maps = m + o_maps;
    g.d_partials = reinterpret_cast<double *>(m + o_part);
    g.d_gbar = reinterpret_cast<unsigned *>(m + o_bar);
    g.d_ctr = reinterpret_cast<unsigned *>(m + o_bar + 64);
    GW_TRY_CUDA(cudaMemcpy(g.d_subs, g.subs.data(), sizeof(SubDev) * nsub, cudaMemcpyHostToDevice));
    GW_TRY_CUDA(cudaMemcpy(g.d_shots, g.shots.data(), sizeof(ShotDev) * nsh, cudaMemcpyHostToDevice));
    GW_TRY_CUDA(cudaMemcpy(g.d_items, g.items.data(), sizeof(Item) * nit, cudaMemcpyHostToDevice));
    size_t off = 0;
    for (gw_domain *d : g.doms) {
        size_t bytes = 128 * kMapsPerSub * (size_t)d->nsub();
        GW_TRY_CUDA(cudaMemcpy(g.d_maps + off, d->d_maps, bytes, cudaMemcpyDeviceToDevice));
        off += bytes;
    }
    GW_TRY_CUDA(cudaMemset(g.d_gbar, 0, 128));           // barrier and tickets
    // the tables are in place before any launch on a non-blocking stream
    GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    g.err = g.doms[0]->d_err;
    return GW_OK;
}

StepArgs group_args(gw_batch *b, Group &g, int k)
{
    StepArgs a{};
    a.subs = g.d_subs;
    a.shots = g.d_shots;
    a.items = g.d_items;
    a.maps = g.d_maps;
    a.partials = g.d_partials;
    a.err = g.err;
    a.seg_base = b->ctx->base;
    a.rank_stride = (long long)b->ctx->rank_bytes;
    a.nitems = (int)g.items.size();
    a.k = k;
    a.nk = 1;
    a.gbar = g.d_gbar;
    a.ctr = g.d_ctr;
    a.dynamic = g.dynamic ? 1 : 0;
    a.symmetric = g.symmetric ? 1 : 0;
    a.fused_halo = g.separate ? 0 : 1;
    return a;
}

}  // namespace

namespace {

// nk steps of one group, then its FP64 norm reduction.
gw_status enqueue_group(gw_batch *b, Group &g, int nk, cudaStream_t s, bool timed,
                        bool count_steps)
{
    // work-item tickets from zero (a launch that gave up may leave them set)
    GW_TRY_CUDA(cudaMemsetAsync(g.d_ctr, 0, sizeof(unsigned), s));
    auto launch = [&](StepArgs a, int steps) -> gw_status {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            GW_TRY_CUDA(cudaEventCreate(&e0));
            GW_TRY_CUDA(cudaEventCreate(&e1));
            GW_TRY_CUDA(cudaEventRecord(e0, s));
        }
        GW_TRY_CUDA(launch_step(b->dtype, g.cfg, g.sponge, g.grid, a, s));
        if (timed) {
            GW_TRY_CUDA(cudaEventRecord(e1, s));
            b->ev.push_back({e0, e1});
            b->ev_steps.push_back(count_steps ? steps : 0);
        }
        return GW_OK;
    };
    if (g.separate) {
        // step, then the face-halo copies of every decomposed member; the
        // copies read the member's step counter like its own launches do
        for (int k = 0; k < nk; ++k) {
            GW_TRY(launch(group_args(b, g, k), 1));
            for (gw_domain *d : g.doms)
                if (!d->halo.empty())
                    GW_TRY_CUDA(launch_halo(d->d_halo, (int)d->halo.size(), d->halo_units,
                                            d->d_subs, d->d_step, k, d->dtype, s));
        }
    } else if (b->persistent && nk > 1) {
        GW_TRY_CUDA(cudaMemsetAsync(g.d_gbar, 0, sizeof(unsigned), s));
        StepArgs a = group_args(b, g, 0);
        a.nk = nk;
        GW_TRY(launch(a, nk));
    } else {
        for (int k = 0; k < nk; ++k) GW_TRY(launch(group_args(b, g, k), 1));
    }
    GW_TRY_CUDA(launch_chunk_end(g.d_shots, (int)g.shots.size(), g.d_partials,
                                 (int)g.items.size(), nk, g.err, s));
    return GW_OK;
}

// One chunk of nk steps of every group on stream s.  Groups of a
// non-persistent batch run side by side on forked streams (different tiles
// mean different kernels; side by side, one group's tail CTAs leave no SM
// idle); persistent groups and timed chunks run one after the other.
gw_status enqueue_all(gw_batch *b, int nk, cudaStream_t s, bool timed)
{
    const size_t ng = b->groups.size();
    if (ng > 1 && !b->persistent && !timed) {
        if (b->aux.size() < ng - 1) {
            if (!b->fork) GW_TRY_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
            while (b->aux.size() < ng - 1) {
                cudaStream_t a = nullptr;
                cudaEvent_t e = nullptr;
                GW_TRY_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
                b->aux.push_back(a);
                GW_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                b->joins.push_back(e);
            }
        }
        GW_TRY_CUDA(cudaEventRecord(b->fork, s));
        for (size_t gi = 1; gi < ng; ++gi) {
            cudaStream_t a = b->aux[gi - 1];
            GW_TRY_CUDA(cudaStreamWaitEvent(a, b->fork, 0));
            GW_TRY(enqueue_group(b, b->groups[gi], nk, a, false, false));
            GW_TRY_CUDA(cudaEventRecord(b->joins[gi - 1], a));
        }
        GW_TRY(enqueue_group(b, b->groups[0], nk, s, false, false));
        for (size_t gi = 1; gi < ng; ++gi)
            GW_TRY_CUDA(cudaStreamWaitEvent(s, b->joins[gi - 1], 0));
        return GW_OK;
    }
    for (size_t gi = 0; gi < ng; ++gi)
        GW_TRY(enqueue_group(b, b->groups[gi], nk, s, timed, gi == 0));
    return GW_OK;
}

gw_status ensure_graph(gw_batch *b)
{
    if (b->gexec) return GW_OK;
    if (!b->cap) GW_TRY_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    GW_TRY_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    gw_status st = enqueue_all(b, b->chunk, b->cap, false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (st != GW_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return GW_OK;
}

void harvest(gw_batch *b)
{
    for (size_t i = 0; i < b->ev.size(); ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, b->ev[i].first, b->ev[i].second) == cudaSuccess)
            b->acc_ms += ms;
        b->acc_n += b->ev_steps[i];
        cudaEventDestroy(b->ev[i].first);
        cudaEventDestroy(b->ev[i].second);
    }
    b->ev.clear();
    b->ev_steps.clear();
}

}  // namespace

extern "C" {

gw_status gw_batch_create(gw_ctx *c, int nshots, gw_domain *const *shots, int chunk,
                          int persistent, gw_batch **out)
{
    if (!c || !shots || nshots <= 0 || !out) return fail(GW_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    if (c->device < 0) return fail(GW_ERR_STATE, "batches need a device context");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    GW_TRY_CUDA(cudaSetDevice(c->device));
    gw_batch *b = new (std::nothrow) gw_batch();
    if (!b) return fail(GW_ERR_NOMEM, "out of host memory");
    b->ctx = c;
    b->dtype = shots[0] ? shots[0]->dtype : 0;
    b->chunk = chunk == 0 ? kDefaultChunk : std::max(1, std::abs(chunk));
    b->graphs = chunk >= 0;
    b->persistent = persistent != 0;
    for (int i = 0; i < nshots; ++i) {
        gw_domain *d = shots[i];
        gw_status st = GW_OK;
        if (!d) st = fail(GW_ERR_ARG, "shot %d is NULL", i);
        else if (d->ctx != c) st = fail(GW_ERR_ARG, "shot %d belongs to another context", i);
        else if (d->dtype != b->dtype) st = fail(GW_ERR_ARG, "shots must share one storage type");
        else if (!d->model_set) st = fail(GW_ERR_STATE, "shot %d has no model", i);
        if (st != GW_OK) {
            delete b;
            return st;
        }
        const bool sponge = d->desc.sponge > 0;
        const bool separate = d->desc.halo_mode == GW_HALO_SEPARATE && !d->halo.empty();
        Group *g = nullptr;
        for (Group &q : b->groups)
            if (q.cfg == d->cfg && q.sponge == sponge && q.symmetric == d->symmetric &&
                q.separate == separate)
                g = &q;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->cfg = d->cfg;
            g->sponge = sponge;
            g->symmetric = d->symmetric;
            g->separate = separate;
            g->ti = d->ti;
        }
        g->doms.push_back(d);
    }
    for (Group &g : b->groups) {
        bool all_static = true;
        for (gw_domain *d : g.doms) all_static = all_static && d->desc.schedule == GW_SCHED_STATIC;
        g.dynamic = !all_static;
    }
    for (Group &g : b->groups) {
        gw_status st = build_group(b, g);
        if (st != GW_OK) {
            gw_batch_destroy(b);
            return st;
        }
    }
    *out = b;
    return GW_OK;
}

gw_status gw_batch_destroy(gw_batch *b)
{
    if (!b) return GW_OK;
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    harvest(b);
    for (Group &g : b->groups)
        if (g.g_meta) ctx_free(b->ctx, g.g_meta);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (cudaStream_t a : b->aux) cudaStreamDestroy(a);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return GW_OK;
}

gw_status gw_batch_step(gw_batch *b, int nsteps, gw_stream stream)
{
    if (!b || nsteps < 0) return fail(GW_ERR_ARG, "bad batch step");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // sources and receivers may have changed through the shots' own calls
    // since the tables were written
    for (Group &g : b->groups) {
        bool dirty = false;
        for (size_t si = 0; si < g.doms.size(); ++si) {
            ShotDev cur = g.doms[si]->shot;
            cur.first_item = g.shots[si].first_item;
            cur.nitems = g.shots[si].nitems;
            if (std::memcmp(&cur, &g.shots[si], sizeof cur) != 0) {
                g.shots[si] = cur;
                dirty = true;
            }
        }
        if (dirty)
            GW_TRY_CUDA(cudaMemcpyAsync(g.d_shots, g.shots.data(),
                                        sizeof(ShotDev) * g.shots.size(),
                                        cudaMemcpyHostToDevice, s));
    }
    int left = nsteps;
    while (left > 0) {
        const bool whole = b->graphs && !b->timing && left >= b->chunk;
        const int nk = whole ? b->chunk : std::min(left, b->chunk);
        if (whole) {
            GW_TRY(ensure_graph(b));
            GW_TRY_CUDA(cudaGraphLaunch(b->gexec, s));
        } else {
            GW_TRY(enqueue_all(b, nk, s, b->timing));
        }
        left -= nk;
    }
    for (Group &g : b->groups)
        for (gw_domain *d : g.doms) {
            // a member with a step limit stops there (its launches skip it)
            d->step = (int)std::min<long long>((long long)d->step + nsteps, d->shot.limit);
            d->last = s;
        }
    return GW_OK;
}

gw_status gw_batch_info(gw_batch *b, int *groups, int *ctas, int *items)
{
    if (!b) return fail(GW_ERR_ARG, "batch is NULL");
    int c = 0, it = 0;
    for (Group &g : b->groups) {
        c += g.grid;
        it += (int)g.items.size();
    }
    if (groups) *groups = (int)b->groups.size();
    if (ctas) *ctas = c;
    if (items) *items = it;
    return GW_OK;
}

gw_status gw_batch_timing(gw_batch *b, int enable)
{
    if (!b) return fail(GW_ERR_ARG, "batch is NULL");
    b->timing = enable != 0;
    return GW_OK;
}

gw_status gw_batch_stats_get(gw_batch *b, gw_kernel_stats *out)
{
    if (!b || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    GW_TRY_CUDA(cudaSetDevice(b->ctx->device));
    GW_TRY_CUDA(cudaDeviceSynchronize());
    harvest(b);
    out->launches = b->acc_n;
    out->total_ms = b->acc_ms;
    out->halo_ms = 0;
    b->acc_n = 0;
    b->acc_ms = 0;
    return GW_OK;
}

}  // extern "C"

extern "C" gw_status gw_pick_tile(int dtype, int nx, int ny, int *tile)
{
    if (!tile || dtype < 0 || dtype > 3 || nx <= 0 || ny <= 0)
        return fail(GW_ERR_ARG, "bad tile-model arguments");
    *tile = step_cfg_pick(dtype, nx, ny) + 1;
    return GW_OK;
}

extern "C" gw_status gw_tile_count(int dtype, int *count)
{
    if (!count || dtype < 0 || dtype > 3) return fail(GW_ERR_ARG, "bad storage type");
    *count = step_cfg_count(dtype);
    return GW_OK;
}

extern "C" gw_status gw_autotune(gw_ctx *c, const gw_shot_desc *desc, int px, int py,
                                 int pz, int steps, int *best_tile, double *best_ms,
                                 double *ms_all, int n_all)
{
    if (!c || !desc || !best_tile || steps <= 0 || n_all < 0 || (n_all > 0 && !ms_all))
        return fail(GW_ERR_ARG, "bad autotune arguments");
    if (desc->dtype < 0 || desc->dtype > 3) return fail(GW_ERR_ARG, "bad storage type");
    if (c->device < 0) return fail(GW_ERR_STATE, "autotuning needs a device context");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    char key[160];
    std::snprintf(key, sizeof key, "%d,%d,%d|%d,%d,%d|%d|%d|%d", desc->nx, desc->ny, desc->nz,
                  px, py, pz, desc->dtype, desc->halo_mode, desc->sponge > 0);
    const int ncfg = step_cfg_count(desc->dtype);
    auto hit = c->tuned.find(key);
    if (hit == c->tuned.end()) {
        const int warm = 3;
        gw_shot_desc dd = *desc;
        dd.nsteps = warm + steps;
        dd.persistent = 0;
        dd.dt = 0;
        // a constant model, set per plane (no host array of the whole grid)
        const std::vector<double> vz((size_t)desc->nz, 2000.0);
        std::vector<double> times(ncfg, 0.0);
        for (int t = 1; t <= ncfg; ++t) {
            dd.tile = t;
            gw_domain *d = nullptr;
            gw_status st = gw_domain_create(c, &dd, px, py, pz, nullptr, nullptr, nullptr, 1, &d);
            if (st != GW_OK) {
                // a tile whose kernel does not fit an SM is skipped; anything
                // else (memory, arguments) is the caller's problem
                if (st == GW_ERR_CUDA && std::strstr(gw_last_error(), "does not fit")) continue;
                return st;
            }
            gw_kernel_stats ks{};
            st = gw_set_model_layered(d, vz.data());
            if (st == GW_OK) st = gw_step(d, warm, nullptr);
            if (st == GW_OK) st = gw_kernel_timing(d, 1);
            if (st == GW_OK) st = gw_step(d, steps, nullptr);
            if (st == GW_OK) st = gw_kernel_stats_get(d, &ks);
            gw_domain_destroy(d);
            if (st != GW_OK) return st;
            times[t - 1] = (ks.total_ms + ks.halo_ms) / std::max(1, ks.launches);
        }
        hit = c->tuned.emplace(key, times).first;
    }
    const std::vector<double> &times = hit->second;
    int best = 0;
    for (int t = 1; t <= ncfg; ++t)
        if (times[t - 1] > 0 && (best == 0 || times[t - 1] < times[best - 1])) best = t;
    if (best == 0) return fail(GW_ERR_CUDA, "no kernel tile fits an SM");
    *best_tile = best;
    if (best_ms) *best_ms = times[best - 1];
    for (int t = 0; t < n_all; ++t) ms_all[t] = t < ncfg ? times[t] : 0.0;
    return GW_OK;
}

extern "C" gw_status gw_plan_tiles(gw_ctx *c, int n, const gw_shot_desc *descs, int steps,
                                   double margin, int *tiles_out)
{
    if (!c || n <= 0 || !descs || !tiles_out || margin < 0)
        return fail(GW_ERR_ARG, "bad tile-planning arguments");
    const int dtype = descs[0].dtype;
    if (dtype < 0 || dtype > 3) return fail(GW_ERR_ARG, "bad storage type");
    const int ncfg = step_cfg_count(dtype);
    std::vector<double> sum(ncfg, 0.0), times(ncfg);
    std::vector<bool> ok(ncfg, true);
    double mixed = 0;
    for (int i = 0; i < n; ++i) {
        if (descs[i].dtype != dtype) return fail(GW_ERR_ARG, "shots must share one storage type");
        // time each tile at full occupancy: the shot's x-y plane over enough
        // planes for 64 M points.  A small shot alone keeps few CTAs busy
        // and times the latency of one CTA's items, not what the tile
        // delivers inside a batch that fills the GPU.  Per point, scaled
        // back to the shot's own planes.
        gw_shot_desc td = descs[i];
        const long long plane = (long long)td.nx * td.ny;
        const long long want = (64LL << 20) / std::max(1LL, plane);
        td.nz = (int)std::max<long long>(td.nz, std::min<long long>(want, 4096));
        int best = 0;
        double bms = 0;
        gw_status st = gw_autotune(c, &td, 1, 1, 1, steps, &best, &bms, times.data(), ncfg);
        if (st == GW_ERR_BUDGET && td.nz != descs[i].nz) {
            // no room in the segment for the taller scratch shot: its own shape
            td = descs[i];
            st = gw_autotune(c, &td, 1, 1, 1, steps, &best, &bms, times.data(), ncfg);
        }
        GW_TRY(st);
        const double scale = (double)descs[i].nz / td.nz;
        for (double &t : times) t *= scale;
        bms *= scale;
        tiles_out[i] = best;
        mixed += bms;
        for (int t = 0; t < ncfg; ++t) {
            if (times[t] <= 0) ok[t] = false;
            sum[t] += times[t];
        }
    }
    int uni = -1;
    for (int t = 0; t < ncfg; ++t)
        if (ok[t] && (uni < 0 || sum[t] < sum[uni])) uni = t;
    if (uni >= 0 && mixed >= (1.0 - margin) * sum[uni])
        for (int i = 0; i < n; ++i) tiles_out[i] = uni + 1;
    return GW_OK;
}
