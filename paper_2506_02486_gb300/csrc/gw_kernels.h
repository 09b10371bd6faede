// gw_kernels.h -- host-side launch interface of the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "gw_device.h"

namespace gw {

// Storage types (same values as the public GW_* dtype codes).
enum Dtype { DT_F32 = 0, DT_F64 = 1, DT_F16S = 2, DT_BF16 = 3 };

inline int dtype_size(int dt) { return dt == DT_F64 ? 8 : dt == DT_F32 ? 4 : 2; }
// Interior x offset in a padded row: >= R and 32-byte (sector) aligned.
inline int dtype_xoff(int dt) { return dtype_size(dt) == 2 ? 16 : dtype_size(dt) == 4 ? 8 : 4; }
// x halo staged in shared memory: >= R and a multiple of 16 bytes.
inline int dtype_halo(int dt) { return dtype_size(dt) == 2 ? 8 : 4; }

struct TileInfo {
    int tx, ty;        // tile extent in x and y (interior points)
    int threads;       // threads per CTA
    size_t smem;       // dynamic shared memory bytes
    int zcap;          // most planes per work item under the dynamic schedule
    double tail;       // dynamic schedule: cost of the last, uneven round of
                       // items, in item times (the z-chunk cost model)
};

// Tile configurations available for a storage type (ids 0..n-1).
int step_cfg_count(int dtype);
// The tile (id) the shape model expects to move the fewest bytes per point
// for an nx x ny plane: halo overhead of the tile times partial-tile waste.
int step_cfg_pick(int dtype, int nx, int ny);
bool step_cfg_info(int dtype, int cfg, TileInfo *out);
// Max resident CTAs per SM of a configuration (after opting in to its
// shared memory); 0 on error.
int step_cfg_occupancy(int dtype, int cfg, bool sponge);

// One launch of the fused step kernel over `grid` CTAs.
cudaError_t launch_step(int dtype, int cfg, bool sponge, int grid,
                        const StepArgs &a, cudaStream_t s);

// ---- auxiliary kernels (aux_kernels.cu) ----

// Max of n doubles (or floats if f32) into *out (as ordered bits; out must
// be zero-initialised before the first call of a reduction).
cudaError_t launch_vmax(const void *v, size_t n, int f32,
                        unsigned long long *out, cudaStream_t s);

// coef = (v * dt / h)^2 in FP64 for a dense slab of planes [z_lo, z_hi) of
// a global model, written into the part of subdomain `sub` inside it.
struct ModelSlab {
    const void *v;     // dense slab, x fastest, (z_hi - z_lo) planes
    int f32;           // v is float (else double)
    int NX, NY;        // global x, y extents
    int z_lo, z_hi;    // global planes in the slab
    double dt_over_h;
    int layered;       // 1: v holds one value per plane (v[z - z_lo])
    int raw;           // 1: store v itself (rounded to the coef type)
};
cudaError_t launch_coef(const ModelSlab &m, const SubDev &sub, int dtype,
                        cudaStream_t s);
// out[i] = in[i] rounded to FP32 (nearest, ties to even) by the integer
// conversion the FP32 coefficient precompute uses.
cudaError_t launch_round_to_f32(const double *in, float *out, size_t n, cudaStream_t s);
// In place over a subdomain whose coef array holds velocities (stored by a
// raw launch_coef): coef = (v dt / h)^2 in FP64, rounded to the coef type.
cudaError_t launch_coef_square(const SubDev &sub, int dtype, double dt_over_h,
                               cudaStream_t s);

// Dense <-> padded transfers of a slab of planes of one field.
// which: 0 = u[cur], 1 = u[cur^1], 2 = w, 3 = coef.  `scale` multiplies on
// scatter and divides on gather (FP16 scaling).
struct FieldSlab {
    void *dense;       // dense slab, x fastest
    int f64;           // dense is double (else float)
    int NX, NY;
    int z_lo, z_hi;
    int which, cur;
    double scale;
};
cudaError_t launch_scatter(const FieldSlab &f, const SubDev &sub, int dtype,
                           cudaStream_t s);
cudaError_t launch_gather(const FieldSlab &f, const SubDev &sub, int dtype,
                          cudaStream_t s);

// Face-halo copy descriptors: R planes of `src` sub into the halo of `dst`.
struct HaloDesc {
    int src, dst;      // subdomain indices
    int face;          // face of src that is copied (0..5: -x,+x,-y,+y,-z,+z)
    int pad_;
    long long first;   // prefix offset of this descriptor's elements
};
// Copy all face halos for descriptors [0, ndesc); max_units = the largest
// number of 16-byte units (rows cut into pieces of 16 / element-size
// elements) of any one face.  The buffer refreshed is u[(*step + k + 1) & 1]:
// the new field after step k of the current chunk, or (k = -1) the current
// field u_n.
cudaError_t launch_halo(const HaloDesc *descs, int ndesc, long long max_units,
                        const SubDev *subs_dev, const int *step, int k,
                        int dtype, cudaStream_t s);

// End of a chunk of `nk` steps: reduce the per-item norm partials in FP64
// (fixed order) into each shot's norm log, flag non-finite values, and
// advance every shot's step counter by nk.
cudaError_t launch_chunk_end(const ShotDev *shots_dev, int nshots,
                             const double *partials, int nitems, int nk,
                             unsigned *err, cudaStream_t s);

// FP64 check reductions over subdomain `sub` of a shot's current state
// (cur = index of the buffer holding u_n; the other holds u_{n-1}):
// Per interior plane z of `sub`: part[3z] = sum u_n^2, part[3z+1] =
// sum (u_n - u_{n-1})^2 / coef, part[3z+2] = sum u_n lap(u_{n-1}); u
// unscaled by 1/scale_u.  launch_check_sum adds nplanes such triples in a
// fixed order into out[0..2].
cudaError_t launch_check(const SubDev &sub, int cur, int dtype,
                         double scale_u, double *part, cudaStream_t s);
cudaError_t launch_check_sum(const double *part, int nplanes, double *out,
                             cudaStream_t s);

// ---- tensor-core block products (gemm_tc.cu) ----

// Bound of the block-product kernel's waits in normal launches (the same
// 4 s as the step kernel's device-side limit).
constexpr unsigned long long kWaitLimitNsHost = 4000000000ull;

// C_q = A_q B_q^T for up to kGemmMaxProb problems of one shape: A_q is an
// m x k BF16 stripe and B_q an n x k BF16 stripe (both K contiguous), read
// through 3-D tensor maps {k, rows, rank} (128-byte swizzle; boxes 64 x
// tile_m for A, 64 x 256 for B); C_q is m x n FP32 at c + c_off[q], row
// pitch ldc.
constexpr int kGemmMaxProb = 64;
struct GemmArgs {
    int nprob;
    int k, m, n;
    int a_rank[kGemmMaxProb];       // rank coordinate of problem q's A stripe
    int b_rank[kGemmMaxProb];       // rank coordinate of its B stripe
    long long c_off[kGemmMaxProb];  // element offset of its block in c
    float *c;
    long long ldc;
    int group;                      // tile rows per raster group
    unsigned *err;                  // ERRB_TIMEOUT when a wait gave up
    unsigned long long wait_ns;     // bound of every wait (kWaitLimitNs normally)
    int skip_loads;                 // self-test: issue no loads, so the waits run out
};
int gemm_tile_n();
// tile_m: rows of one CTA's output tile, 128 (4 stages of 48 KB, two
// accumulators) or 256 (3 stages of 64 KB, one accumulator pair).  Most
// CTAs resident at once (one per SM); 0 on error.
int gemm_max_ctas(int tile_m, int num_sms);
// map_a / map_b: host copies of the encoded tensor maps (CUtensorMap) with
// a box of 64 elements along K and tile_m A rows or 256 B rows.  grid:
// CTAs, at most gemm_max_ctas.
cudaError_t launch_gemm_bf16(const void *map_a, const void *map_b, const GemmArgs &a,
                             int tile_m, int grid, cudaStream_t s);

}  // namespace gw
