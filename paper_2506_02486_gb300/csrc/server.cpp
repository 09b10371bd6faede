// server.cpp -- continuous-batching shot server.  One loop thread owns all
// GPU work: it admits submitted shots in arrival order while they fit the
// HBM budget and a slot, sets them up (legacy-stream copies, overlapped
// with the running chunk), advances every resident shot with one multi-shot
// batch per storage type, each on a non-blocking stream of its own (tile
// groups side by side within it), and retires shots
// at chunk boundaries (traces to the caller's buffer, final check).
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "domain_impl.h"

using namespace gw;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    gw_request r{};
    std::vector<double> vz;      // owned copy of a layered model
    std::vector<int> rec;        // owned copy of the receivers
    size_t bytes = 0;            // footprint charged against the budget
    long long points = 0;
    gw_result res{};
    gw_domain *dom = nullptr;
    int left = 0;                // steps still to take
};

}  // namespace

struct gw_server {
    gw_ctx *ctx = nullptr;
    size_t budget = 0;
    int slots = 0;
    int chunk = kDefaultChunk;
    cudaStream_t streams[4] = {nullptr, nullptr, nullptr, nullptr};  // one per storage type
    cudaStream_t aux = nullptr;  // reading finished shots while a chunk runs
    Clock::time_point t0;
    std::thread th;

    // shared with the callers, under mu
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> live;   // pending or active
    std::unordered_map<uint64_t, Req *> done;   // completed, not yet waited
    uint64_t next = 1;
    bool stop = false;
    bool blocked = false;        // the head did not fit the segment: wait for a retirement
    size_t used = 0;
    gw_server_stats st{};

    // loop thread only
    std::vector<Req *> active;
    std::vector<Req *> retiring;   // finished in the last chunk, not yet read
    std::vector<std::pair<gw_domain *, size_t>> grave;   // read; freed after the chunk
    gw_batch *batch[4] = {nullptr, nullptr, nullptr, nullptr};

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
};

namespace {

// Pop the admissible prefix of the queue (arrival order: a shot that does
// not fit holds back the ones behind it, so large shots are not starved).
void take_admissible(gw_server *S, std::vector<Req *> &out)
{
    while (!S->pending.empty() && !S->blocked) {
        Req *q = S->pending.front();
        const int resident = (int)(S->active.size() + out.size());
        if (resident >= S->slots || S->used + q->bytes > S->budget) break;
        S->pending.pop_front();
        S->used += q->bytes;
        S->st.peak_bytes = std::max(S->st.peak_bytes, S->used);
        out.push_back(q);
    }
}

// The result is ready: gw_wait hands it out (and frees q).  The shot's
// domain and its share of the budget go separately (release), so that a
// shot can be completed while the next chunk runs and freed once no launch
// covers it any more.
void complete(gw_server *S, Req *q, gw_status status)
{
    std::lock_guard<std::mutex> lk(S->mu);
    q->res.status = status;
    q->res.done_s = S->now();
    S->live.erase(q->ticket);
    S->done[q->ticket] = q;
    S->st.completed++;
    S->cv_done.notify_all();
}

void release(gw_server *S, gw_domain *dom, size_t bytes)
{
    if (dom) gw_domain_destroy(dom);
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= bytes;
    S->blocked = false;
}

void finish(gw_server *S, Req *q, gw_status status)
{
    gw_domain *dom = q->dom;
    const size_t bytes = q->bytes;
    q->dom = nullptr;
    complete(S, q, status);
    release(S, dom, bytes);
}

// Create the shot's domain and load its model, source and receivers.
gw_status setup(gw_server *S, Req *q)
{
    q->res.admit_s = S->now();
    gw_shot_desc d = q->r.desc;
    if (d.tile == 0) GW_TRY(gw_pick_tile(d.dtype, d.nx, d.ny, &d.tile));
    GW_TRY(gw_domain_create(S->ctx, &d, 1, 1, 1, nullptr, nullptr, nullptr, 1, &q->dom));
    if (q->r.vel) GW_TRY(gw_set_model_f32(q->dom, q->r.vel));
    else GW_TRY(gw_set_model_layered(q->dom, q->vz.data()));
    GW_TRY(gw_inject_ricker(q->dom, q->r.src[0], q->r.src[1], q->r.src[2], q->r.f_peak));
    if (q->r.nrec) GW_TRY(gw_set_receivers(q->dom, q->r.nrec, q->rec.data()));
    q->res.tile = q->dom->cfg + 1;
    q->left = d.nsteps;
    // the shot stops at its own step count inside a longer chunk of the
    // batch (its launches skip it from there on)
    q->dom->shot.limit = d.nsteps;
    return GW_OK;
}

// Set up newly admitted shots; those that cannot be placed in the segment
// (fragmentation) go back to the head of the queue while others are
// resident.  Returns the shots ready to join.
std::vector<Req *> setup_all(gw_server *S, std::vector<Req *> &adm, bool others_resident)
{
    std::vector<Req *> ready;
    for (size_t i = 0; i < adm.size(); ++i) {
        Req *q = adm[i];
        gw_status st = setup(S, q);
        if (st == GW_OK) {
            ready.push_back(q);
            continue;
        }
        if (q->dom) {
            gw_domain_destroy(q->dom);
            q->dom = nullptr;
        }
        if (st == GW_ERR_BUDGET && (others_resident || !ready.empty())) {
            std::lock_guard<std::mutex> lk(S->mu);
            // this one and every later admission go back, in order
            for (size_t j = adm.size(); j-- > i;) {
                if (adm[j]->dom) {
                    gw_domain_destroy(adm[j]->dom);
                    adm[j]->dom = nullptr;
                }
                S->pending.push_front(adm[j]);
                S->used -= adm[j]->bytes;
            }
            S->blocked = true;
            break;
        }
        finish(S, q, st);
    }
    adm.clear();
    return ready;
}

gw_status rebuild(gw_server *S)
{
    for (gw_batch *&b : S->batch) {
        if (b) gw_batch_destroy(b);
        b = nullptr;
    }
    for (int t = 0; t < 4; ++t) {
        std::vector<gw_domain *> doms;
        for (Req *q : S->active)
            if (q->r.desc.dtype == t) doms.push_back(q->dom);
        if (doms.empty()) continue;
        // plain per-step launches, tile groups side by side: membership
        // changes too often for captured graphs to pay off, and persistent
        // (cooperative) groups would have to run one after the other
        GW_TRY(gw_batch_create(S->ctx, (int)doms.size(), doms.data(), -S->chunk, 0,
                               &S->batch[t]));
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.rebuilds++;
    return GW_OK;
}

// A finished shot's traces and final check (the sums of gw_check, by the
// same kernels) on the server's own stream: no launch of the running chunk
// covers the shot any more, so this waits for nothing else on the device
// (gw_read_receivers and gw_check would wait for the whole device).
gw_status collect(gw_server *S, Req *q)
{
    gw_domain *d = q->dom;
    cudaStream_t s = S->aux;
    unsigned err = 0;
    double a[3] = {0.0, 0.0, 0.0};
    GW_TRY_CUDA(cudaMemcpyAsync(&err, d->d_err, sizeof err, cudaMemcpyDeviceToHost, s));
    const int n = q->r.desc.nsteps;
    if (q->r.traces && q->r.nrec)
        GW_TRY_CUDA(cudaMemcpy2DAsync(q->r.traces, sizeof(float) * n, d->d_traces,
                                      sizeof(float) * d->shot.cap, sizeof(float) * n,
                                      q->r.nrec, cudaMemcpyDeviceToHost, s));
    int planes = 0;
    for (const SubDev &sd : d->subs) {
        GW_TRY_CUDA(launch_check(sd, d->step & 1, d->dtype, d->su, d->d_chk + 3 * planes, s));
        planes += sd.nz;
    }
    GW_TRY_CUDA(launch_check_sum(d->d_chk, planes, d->d_scratch, s));
    GW_TRY_CUDA(cudaMemcpyAsync(a, d->d_scratch, sizeof a, cudaMemcpyDeviceToHost, s));
    GW_TRY_CUDA(cudaStreamSynchronize(s));
    if (err & ERRB_TIMEOUT) return fail(GW_ERR_TIMEOUT, "a device wait gave up (error bits 0x%x)", err);
    if (err & ERRB_NONFINITE) return fail(GW_ERR_NUMERIC, "non-finite wavefield norm (error bits 0x%x)", err);
    if (err) return fail(GW_ERR_STATE, "device error bits 0x%x", err);
    q->res.norm2 = a[0];
    q->res.energy = a[1] - a[2];
    if (!std::isfinite(a[0]) || !std::isfinite(a[1]) || !std::isfinite(a[2]))
        return fail(GW_ERR_NUMERIC, "non-finite check reduction");
    return GW_OK;
}

// Complete the shots that finished in the last chunk; their domains go to
// the grave (freed after the next chunk) or, with nothing running, at once.
void retire_all(gw_server *S, bool now)
{
    for (Req *q : S->retiring) {
        const gw_status st = collect(S, q);
        gw_domain *dom = q->dom;
        const size_t bytes = q->bytes;
        q->dom = nullptr;
        complete(S, q, st);
        if (now) release(S, dom, bytes);
        else S->grave.push_back({dom, bytes});
    }
    S->retiring.clear();
}

void free_grave(gw_server *S)
{
    for (auto &g : S->grave) release(S, g.first, g.second);
    S->grave.clear();
}

void loop(gw_server *S)
{
    cudaSetDevice(S->ctx->device);
    bool dirty = false;
    for (;;) {
        std::vector<Req *> adm;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->active.empty() && S->retiring.empty()) {
                S->cv_work.wait(lk, [&] {
                    return S->stop || (!S->pending.empty() && !S->blocked);
                });
            }
            if (S->stop) break;
            take_admissible(S, adm);
        }
        if (!adm.empty()) {
            std::vector<Req *> ready = setup_all(S, adm, !S->active.empty());
            if (!ready.empty()) {
                S->active.insert(S->active.end(), ready.begin(), ready.end());
                dirty = true;
            }
        }
        if (S->active.empty()) {
            // nothing to run beside it: finish the last shots now
            retire_all(S, true);
            continue;
        }
        if (dirty) {
            gw_status st = rebuild(S);
            if (st != GW_OK) {
                for (Req *q : S->active) finish(S, q, st);
                S->active.clear();
                continue;
            }
            dirty = false;
        }
        // chunks of K steps for every member; a member with fewer steps
        // left stops at its limit inside the chunk, so K is set by the
        // member with the most steps left (at most the server's chunk)
        int K = 1;
        long long pts = 0;
        for (Req *q : S->active) K = std::max(K, std::min(S->chunk, q->left));
        for (Req *q : S->active) pts += q->points * std::min(K, q->left);
        const double t_launch = S->now();
        gw_status st = GW_OK;
        // the storage types' batches run side by side, one stream each
        for (int t = 0; t < 4; ++t)
            if (S->batch[t] && st == GW_OK) st = gw_batch_step(S->batch[t], K, S->streams[t]);
        // while the chunk runs: complete the shots of the last chunk, admit
        // and set up the next ones
        retire_all(S, false);
        std::vector<Req *> joiners;
        if (st == GW_OK) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                take_admissible(S, adm);
            }
            if (!adm.empty()) joiners = setup_all(S, adm, true);
        }
        cudaError_t e = cudaSuccess;
        for (cudaStream_t x : S->streams) {
            cudaError_t ex = cudaStreamSynchronize(x);
            if (e == cudaSuccess) e = ex;
        }
        if (st == GW_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.chunks++;
            S->st.point_updates += pts;
            S->st.busy_s += S->now() - t_launch;
        }
        // no launch covers the shots completed during this chunk any more
        free_grave(S);
        std::vector<Req *> keep;
        for (Req *q : S->active) {
            if (st != GW_OK) {
                finish(S, q, st);
                dirty = true;
                continue;
            }
            q->left -= K;
            if (q->left > 0) {
                keep.push_back(q);
            } else {
                // read during the next chunk (or at once if none runs)
                S->retiring.push_back(q);
                dirty = true;
            }
        }
        S->active.swap(keep);
        if (!joiners.empty()) {
            S->active.insert(S->active.end(), joiners.begin(), joiners.end());
            dirty = true;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.max_active = std::max(S->st.max_active, (int)S->active.size());
    }
    // stopped: nothing runs any more
    for (cudaStream_t x : S->streams) cudaStreamSynchronize(x);
    free_grave(S);
    retire_all(S, true);
    for (gw_batch *&b : S->batch) {
        if (b) gw_batch_destroy(b);
        b = nullptr;
    }
    for (Req *q : S->active) finish(S, q, GW_ERR_STATE);
    S->active.clear();
    std::vector<Req *> rest;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        rest.assign(S->pending.begin(), S->pending.end());
        S->pending.clear();
    }
    for (Req *q : rest) finish(S, q, GW_ERR_STATE);
}

}  // namespace

extern "C" {

gw_status gw_server_create(gw_ctx *c, size_t hbm_budget, int max_slots, int chunk,
                           gw_server **out)
{
    if (!c || !out || hbm_budget == 0 || max_slots <= 0 || chunk < 0)
        return fail(GW_ERR_ARG, "bad server arguments");
    *out = nullptr;
    if (c->device < 0) return fail(GW_ERR_STATE, "serving needs a device context");
    if (!c->base) return fail(GW_ERR_STATE, "no segment attached");
    if (hbm_budget > c->rank_bytes)
        return fail(GW_ERR_BUDGET, "budget of %zu bytes exceeds the segment (%zu per rank)",
                    hbm_budget, c->rank_bytes);
    gw_server *S = new (std::nothrow) gw_server();
    if (!S) return fail(GW_ERR_NOMEM, "out of host memory");
    S->ctx = c;
    S->budget = hbm_budget;
    S->slots = max_slots;
    S->chunk = chunk == 0 ? kDefaultChunk : chunk;
    S->st.budget_bytes = hbm_budget;
    cudaError_t e = cudaSetDevice(c->device);
    for (int t = 0; t < 4 && e == cudaSuccess; ++t)
        e = cudaStreamCreateWithFlags(&S->streams[t], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaStream_t x : S->streams)
            if (x) cudaStreamDestroy(x);
        delete S;
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    S->t0 = Clock::now();
    try {
        S->th = std::thread(loop, S);
    } catch (...) {
        for (cudaStream_t x : S->streams)
            if (x) cudaStreamDestroy(x);
        cudaStreamDestroy(S->aux);
        delete S;
        return fail(GW_ERR_NOMEM, "cannot start the server thread");
    }
    *out = S;
    return GW_OK;
}

gw_status gw_server_destroy(gw_server *S)
{
    if (!S) return GW_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->done) delete kv.second;
    for (cudaStream_t x : S->streams)
        if (x) cudaStreamDestroy(x);
    if (S->aux) cudaStreamDestroy(S->aux);
    delete S;
    return GW_OK;
}

gw_status gw_submit(gw_server *S, const gw_request *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) return fail(GW_ERR_ARG, "NULL argument");
    const gw_shot_desc &D = req->desc;
    if (D.nx <= 0 || D.ny <= 0 || D.nz <= 0 || D.nsteps <= 0)
        return fail(GW_ERR_ARG, "a request needs a grid and at least one step");
    if (!req->vel && !req->vz) return fail(GW_ERR_ARG, "a request needs vel or vz");
    if (req->nrec < 0 || (req->nrec && !req->rec)) return fail(GW_ERR_ARG, "bad receivers");
    size_t bytes = 0;
    GW_TRY(gw_domain_bytes(&D, 1, 1, 1, req->nrec, &bytes));
    if (bytes > S->budget)
        return fail(GW_ERR_BUDGET, "shot needs %zu bytes; the budget is %zu", bytes, S->budget);
    Req *q = new (std::nothrow) Req();
    if (!q) return fail(GW_ERR_NOMEM, "out of host memory");
    q->r = *req;
    if (!req->vel) q->vz.assign(req->vz, req->vz + D.nz);
    q->r.vz = nullptr;
    if (req->nrec) q->rec.assign(req->rec, req->rec + 3 * (size_t)req->nrec);
    q->r.rec = nullptr;
    q->bytes = bytes;
    q->points = (long long)D.nx * D.ny * D.nz;
    q->res.steps = D.nsteps;
    q->res.points = q->points;
    q->res.device_bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete q;
            return fail(GW_ERR_STATE, "server is stopping");
        }
        q->ticket = S->next++;
        q->res.submit_s = S->now();
        S->pending.push_back(q);
        S->live[q->ticket] = q;
        *ticket = q->ticket;
    }
    S->cv_work.notify_all();
    return GW_OK;
}

gw_status gw_wait(gw_server *S, uint64_t ticket, int timeout_ms, gw_result *out)
{
    if (!S || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return S->done.count(ticket) || !S->live.count(ticket); };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return fail(GW_ERR_TIMEOUT, "ticket %llu not complete", (unsigned long long)ticket);
    }
    auto it = S->done.find(ticket);
    if (it == S->done.end())
        return fail(GW_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    *out = it->second->res;
    delete it->second;
    S->done.erase(it);
    return GW_OK;
}

gw_status gw_server_stats_get(gw_server *S, gw_server_stats *out)
{
    if (!S || !out) return fail(GW_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->pending = (int)S->pending.size();
    out->active = (int)(S->live.size() - S->pending.size());
    out->used_bytes = S->used;
    out->now_s = S->now();
    return GW_OK;
}

double gw_server_now(gw_server *S) { return S ? S->now() : 0.0; }

}  // extern "C"
