// domain_impl.h -- the host object behind gw_domain (shared by the domain
// runtime and the multi-shot batch).
#pragma once
#include <cuda.h>

#include <utility>
#include <vector>

#include "gw_internal.h"

namespace gw {
constexpr int kDefaultChunk = 25;

// Tile columns (ti.tx x ti.ty) of all of `subs`.
long long tile_columns(const std::vector<SubDev> &subs, const TileInfo &ti);
// The work-item schedule of a shot: `sched` (GW_SCHED_*) if it forces one,
// else static for an undecomposed shot whose tile columns fit in one round
// of `grid` CTAs and dynamic otherwise.
bool dynamic_schedule(int sched, int nsub, long long ncols, int grid);
// Work items of `subs` (subdomain indices offset by sub_base) for a tile of
// ti.tx x ti.ty, z-chunk-major; zchunk <= 0 lets the cost model pick the
// planes per item for `grid` CTAs under the schedule `sched` would give
// (tail_hidden: other launches run beside this one and fill its last
// round, so the items only need to be long).  Returns the planes per item
// used.
int make_items(const std::vector<SubDev> &subs, const TileInfo &ti, int grid,
               int zchunk, int sched, std::vector<Item> &items, int sub_base = 0,
               bool tail_hidden = false);
}  // namespace gw

using gw::HaloDesc;
using gw::Item;
using gw::ShotDev;
using gw::SubDev;
using gw::TileInfo;

struct gw_domain {
    gw_ctx *ctx = nullptr;
    gw_shot_desc desc{};
    int dtype = gw::DT_F32;
    bool delta = false;
    int np[3] = {1, 1, 1};
    bool symmetric = true;
    std::vector<int> split[3];
    std::vector<SubDev> subs;
    std::vector<gw_gptr> allocs;          // every allocation we own
    gw_gptr g_fields[4] = {0, 0, 0, 0};   // u0, u1, w, coef
    size_t device_bytes = 0;
    // device metadata
    SubDev *d_subs = nullptr;
    ShotDev *d_shot = nullptr;
    char *d_maps = nullptr;
    unsigned *d_err = nullptr;
    int *d_step = nullptr;
    unsigned *d_gbar = nullptr;           // barrier of persistent launches
    unsigned *d_ctr = nullptr;            // work-item tickets of the step kernel
    bool dynamic = false;                 // dynamic work-item schedule
    double *d_scratch = nullptr;          // 4 doubles for checks
    double *d_chk = nullptr;              // 3 per-plane check partials per z
    double *d_wavelet = nullptr;
    double *d_norms = nullptr;
    double *d_gtab = nullptr;             // gx | gy | gz
    int4 *d_src = nullptr;
    int4 *d_rec = nullptr;
    float *d_traces = nullptr;
    Item *d_items = nullptr;
    double *d_partials = nullptr;
    HaloDesc *d_halo = nullptr;
    gw_gptr g_rec = 0, g_traces = 0, g_items = 0;
    ShotDev shot{};
    // schedule
    int cfg = 0;
    TileInfo ti{};
    int grid = 0, nitems = 0, chunk = gw::kDefaultChunk, zc = 0;
    std::vector<Item> items;
    std::vector<HaloDesc> halo;
    long long halo_units = 0;
    // sources and receivers (host copies)
    std::vector<int4> srcs;
    std::vector<int4> recs;               // receivers (host copy)
    std::vector<std::vector<double>> wavelets;
    int nrec = 0;
    // model
    double dt = 0, vmax = 0, courant = 0;
    bool model_set = false;
    double su = 1, sw = 1;
    int step = 0;                         // steps enqueued
    cudaStream_t last = nullptr;
    // graphs
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_step, ev_halo;
    std::vector<int> ev_steps;            // steps covered by each ev_step pair
    double acc_ms = 0, acc_halo_ms = 0;
    int acc_n = 0;

    int nsub() const { return (int)subs.size(); }
    int esize() const { return gw::dtype_size(dtype); }
};
