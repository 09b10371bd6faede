/*
 * gbwave.h -- C ABI of the GB300 (sm_103a) Minimod acoustic-isotropic
 * library: PGAS-style global memory, subdomain halo put / fence, and the
 * fused 25-point-stencil leapfrog time step.
 *
 * Paper: "DiOMP-Offloading: Toward Portable Distributed Heterogeneous
 * OpenMP" (arXiv 2506.02486).  Section 3.2 defines the global segment with
 * symmetric and asymmetric allocation (32-byte second-level pointers and a
 * remote-pointer cache); Listing 1 (section 4.5) is the Minimod halo
 * exchange: every rank puts its boundary slabs into its neighbours with a
 * one-sided device-to-device put, then fences.  Here the "ranks" are the
 * subdomains of one grid, all resident in one GPU's HBM, and a put is a
 * device store into the neighbour's halo.
 *
 * The numerical scheme (not printed in the paper, which names only the
 * "acoustic isotropic kernel" of Minimod, section 4.5):
 *
 *   lap(u)  = sum over x, y, z of c0 u + sum_{m=1..4} c_m (u[-m] + u[+m]),
 *             c = (-205/72, 8/5, -1/5, 8/315, -1/560)
 *   u_{n+1} = G (2 u_n - G u_{n-1} + coef (lap(u_n) + src_n)),
 *   coef    = (v dt / h)^2,   G = g_x g_y g_z (Cerjan sponge),
 *   src_n   = wavelet[n] at the source cell(s), 0 elsewhere.
 *
 * Conventions for every entry point:
 *   - Return value: GW_OK (0) or a negative GW_ERR_* code; nothing aborts.
 *     gw_last_error() gives a message for the calling thread.
 *   - Device work is enqueued on the gw_stream argument (a cudaStream_t;
 *     NULL = the legacy default stream) and is asynchronous unless the
 *     entry point says it synchronises.  Faults found by kernels (a wait
 *     that gave up, a non-finite norm) are latched in a device error word
 *     and reported by the next synchronising call.
 *   - Host arrays are owned by the caller and only read/written during the
 *     call.  Interior host arrays are x fastest, then y, then z
 *     (index (z*ny + y)*nx + x), with no halo.
 *   - The global segment is device memory owned by the caller (e.g. a
 *     PyTorch tensor); the library sub-allocates it and owns only its
 *     own metadata.  Destroy domains before releasing the segment.
 */
#ifndef GBWAVE_H
#define GBWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gw_status;
#define GW_OK            0
#define GW_ERR_ARG      -1   /* invalid argument                          */
#define GW_ERR_BUDGET   -2   /* does not fit the segment / HBM budget     */
#define GW_ERR_ALIGN    -3   /* pointer or size misaligned                */
#define GW_ERR_CUDA     -4   /* a CUDA runtime call failed                */
#define GW_ERR_TIMEOUT  -5   /* a bounded device or host wait gave up     */
#define GW_ERR_STATE    -6   /* call not valid in the object's state      */
#define GW_ERR_NUMERIC  -7   /* a check reduction found a non-finite value */
#define GW_ERR_NOMEM    -8   /* host allocation failed                    */

typedef struct gw_ctx gw_ctx;
typedef struct gw_domain gw_domain;
typedef struct gw_batch gw_batch;
typedef struct gw_server gw_server;
typedef void *gw_stream;          /* cudaStream_t */
typedef uint64_t gw_gptr;         /* handle of a global allocation; 0 = none */

/* Storage types of the wavefields.  Arithmetic is FP32 for GW_F32,
 * GW_F16S and GW_BF16, FP64 for GW_F64.  GW_F16S stores FP16 scaled by a
 * per-shot power of two; the reduced types use the delta form
 * w_n = u_n - G u_{n-1}:  w' = G (w + coef (lap(u) + src)),  u' = G u + w'
 * (algebraically the same recurrence: u' = G u + G (u - G u_{n-1} +
 * coef (lap + src)) = G (2u - G u_{n-1} + coef (lap + src)); only the
 * rounding of the stored values differs). */
enum { GW_F32 = 0, GW_F64 = 1, GW_F16S = 2, GW_BF16 = 3 };

/* How the halo of each subdomain is refreshed after a step. */
enum {
    GW_HALO_FUSED = 0,     /* the step kernel stores boundary values straight
                              into the neighbours' halos (one-sided put in
                              the epilogue); fence = kernel boundary      */
    GW_HALO_SEPARATE = 1   /* a pack/put/unpack kernel after each step    */
};

/* Fields readable/writable through gw_read_wavefield / gw_write_wavefield. */
enum {
    GW_FIELD_U = 0,        /* u_n, the current wavefield                  */
    GW_FIELD_UPREV = 1,    /* u_{n-1} (3-level storage only)              */
    GW_FIELD_W = 2,        /* w_n = u_n - G u_{n-1} (delta storage only)  */
    GW_FIELD_COEF = 3      /* (v dt / h)^2 as stored                       */
};

/* One shot (one grid).  Zero-initialise and set what you need. */
typedef struct {
    int nx, ny, nz;        /* interior grid points                        */
    double h;              /* grid spacing (m)                            */
    double courant;        /* nu = vmax dt / h; <= 0: half the stability
                              limit, nu = 0.5 * sqrt(4 / (3 |L(pi)|))     */
    double dt;             /* > 0: use this time step, ignore courant     */
    int nsteps;            /* capacity of the wavelet / trace / norm logs */
    int dtype;             /* GW_F32, GW_F64, GW_F16S, GW_BF16            */
    int sponge;            /* Cerjan layer width in cells (0 = none)      */
    double sponge_a;       /* Cerjan constant; <= 0: 0.015                */
    int periodic;          /* bit 0: x, bit 1: y, bit 2: z wrap around    */
    int halo_mode;         /* GW_HALO_FUSED or GW_HALO_SEPARATE           */
    int chunk;             /* steps per CUDA-graph chunk; 0: 25; < 0: no
                              graphs (plain launches)                     */
    int tile;              /* kernel tile configuration id + 1; 0: default */
    int zchunk;            /* planes per work item; 0: chosen by the cost
                              model (load balance vs z-halo re-reads; at
                              least two z-chunks per column, at most 512
                              planes)                                     */
    double scale_u;        /* GW_F16S: power-of-two scale of u; 0: auto   */
    double scale_w;        /* GW_F16S: power-of-two scale of w; 0: auto   */
    int persistent;        /* != 0: each chunk of steps is one launch whose
                              CTAs wait for each other between steps (a
                              bounded device-wide barrier; cooperative
                              launch); needs GW_HALO_FUSED                */
    int schedule;          /* work items to CTAs: GW_SCHED_AUTO (0),
                              GW_SCHED_STATIC or GW_SCHED_DYNAMIC; the same
                              results with every choice                   */
} gw_shot_desc;

/* How a launch's CTAs share the work items of a step.  STATIC: CTA b takes
 * items b, b + grid, ... (balanced when the items are alike and there are
 * few per CTA; CTAs on neighbouring tiles stay in step).  DYNAMIC: the CTAs
 * take the items in order from a shared ticket counter (a CTA held up by a
 * costlier item -- a partial tile, halo puts, sources -- takes fewer).
 * AUTO: STATIC for an undecomposed shot whose tile columns (the x-y tiles
 * of one z-chunk) all fit in one round of CTAs, DYNAMIC otherwise.  Batches
 * use DYNAMIC unless every shot asks for STATIC. */
enum { GW_SCHED_AUTO = 0, GW_SCHED_STATIC = 1, GW_SCHED_DYNAMIC = 2 };

typedef struct {
    double dt;             /* time step used (s)                          */
    double courant;        /* vmax dt / h                                 */
    double vmax;           /* max velocity of the model (0 before set)    */
    int nsub;              /* number of subdomains                        */
    int step;              /* steps taken                                 */
    int tile;              /* kernel tile configuration in use            */
    int ctas;              /* CTAs per step launch                        */
    int items;             /* work items (tile columns x z-chunks)        */
    double scale_u, scale_w;
    size_t device_bytes;   /* segment bytes held by the domain            */
    int schedule;          /* GW_SCHED_STATIC or GW_SCHED_DYNAMIC in use   */
} gw_domain_info;

typedef struct {
    int launches;          /* steps timed (a persistent launch counts each
                              of its steps)                               */
    double total_ms;       /* summed device time of the step kernels      */
    double halo_ms;        /* summed device time of separate halo kernels */
} gw_kernel_stats;

/* ------------------------------------------------------------------ */
/* errors and context                                                  */

/* Message of the last failing call on this thread ("" if none). */
const char *gw_last_error(void);
/* Short name of a status code. */
const char *gw_status_string(gw_status s);
/* Library version string. */
const char *gw_version(void);

/* Create a context on CUDA device `device` (>= 0).  device = -1 creates a
 * host-only context whose "segment" is host memory: allocation, address
 * translation and the pointer cache work, nothing runs on a GPU (used to
 * test the allocator without a GPU). */
gw_status gw_ctx_create(gw_ctx **out, int device);
gw_status gw_ctx_destroy(gw_ctx *ctx);

/* ------------------------------------------------------------------ */
/* global segment and PGAS allocation (paper section 3.2)              */

/* Attach the caller's buffer [base, base + bytes) as the global segment,
 * divided into `nranks` equal per-rank segments (bytes / nranks rounded
 * down to 4 KiB).  base must be 256-byte aligned.  Symmetric allocations
 * grow upward from each rank segment's base at the same offset on every
 * rank; asymmetric data grows downward from each rank segment's end, as in
 * the paper's Figure "memory".  The buffer is zeroed on attach when
 * zero != 0 (device contexts only). */
gw_status gw_segment_attach(gw_ctx *ctx, void *base, size_t bytes,
                            int nranks, int zero);
/* Per-rank bytes, bytes used by symmetric and (max over ranks) asymmetric
 * allocations. */
gw_status gw_segment_info(gw_ctx *ctx, size_t *rank_bytes, size_t *sym_used,
                          size_t *asym_used);

/* Symmetric allocation (section 3.2): every rank gets `bytes` at the same
 * offset, so rank r's block is segment_base(r) + offset.  256-byte aligned.
 * GW_ERR_BUDGET if it does not fit. */
gw_status gw_alloc_symmetric(gw_ctx *ctx, size_t bytes, gw_gptr *out);
/* Asymmetric allocation (section 3.2): rank r gets bytes[r] (nranks
 * entries, zero allowed).  A 32-byte second-level pointer record is
 * allocated symmetrically; rank r's data is placed at the end of its
 * segment and its record is set to point to it.  Record layout (device
 * memory, little-endian): u64 address, u64 bytes, u32 rank, u32 flags,
 * u64 reserved. */
gw_status gw_alloc_asymmetric(gw_ctx *ctx, const size_t *bytes,
                              gw_gptr *out);
/* Free an allocation on every rank; cached translations of it are dropped. */
gw_status gw_free(gw_ctx *ctx, gw_gptr g);
/* Translate (g, rank) to an address in rank's segment.  Symmetric: base of
 * rank + offset.  Asymmetric: the second-level record of that rank is read
 * (one device-to-host fetch) the first time and served from the remote
 * pointer cache afterwards.  bytes (may be NULL) receives the size. */
gw_status gw_resolve(gw_ctx *ctx, gw_gptr g, int rank, void **addr,
                     size_t *bytes);
/* Hits and misses of the remote pointer cache. */
gw_status gw_ptr_cache_stats(gw_ctx *ctx, uint64_t *hits, uint64_t *misses);

/* One-sided put (section 3.2, Listing 1's ompx_put with D2D): copy `bytes`
 * from device address src into rank dst_rank's block of g at byte offset
 * dst_off, on `stream`.  GW_ERR_ARG if out of the block. */
gw_status gw_put(gw_ctx *ctx, gw_gptr dst, int dst_rank, size_t dst_off,
                 const void *src, size_t bytes, gw_stream stream);
/* One-sided get: the mirror of gw_put. */
gw_status gw_get(gw_ctx *ctx, void *dst, gw_gptr src, int src_rank,
                 size_t src_off, size_t bytes, gw_stream stream);
/* Fence (Listing 1's ompx_fence): every put/get issued through this
 * context on any stream, and every non-blocking put/get below, is complete
 * and visible to work enqueued on `stream` afterwards (stream order; no
 * host synchronisation).  The pool streams it joins are released. */
gw_status gw_fence(gw_ctx *ctx, gw_stream stream);

/* Non-blocking one-sided put and get on the context's stream pool (section
 * 3.2: one-sided operations run on pooled streams; "Bounded Concurrency").
 * The copy starts after the work already enqueued on `after` (an event
 * join; the caller's stream is not blocked) and runs on a pool stream, so
 * it overlaps later work on `after`.  It is complete before work enqueued on
 * a stream after gw_fence(ctx, that stream), or on the host after gw_quiet.
 * Same range checks as gw_put / gw_get.  On a host-only context the copy is
 * done at once.
 *
 * Pool policy: streams are created lazily, one per concurrent operation,
 * and reused once released.  At most max_active (default 8) carry
 * unreleased operations.  An operation that finds max_active streams active
 * first makes a partial synchronisation: of the active streams whose work
 * has completed, the oldest half (rounded up) are released and the others
 * keep running; if none has completed, the host waits for the oldest one
 * and releases it. */
gw_status gw_put_nbi(gw_ctx *ctx, gw_gptr dst, int dst_rank, size_t dst_off,
                     const void *src, size_t bytes, gw_stream after);
gw_status gw_get_nbi(gw_ctx *ctx, void *dst, gw_gptr src, int src_rank,
                     size_t src_off, size_t bytes, gw_stream after);
/* Host wait for every non-blocking operation; all pool streams released. */
gw_status gw_quiet(gw_ctx *ctx);
/* The MAX_ACTIVE_STREAMS threshold of section 3.2: 1 .. 64.  A lower value
 * than the current number of active streams takes effect at the next
 * operation, which releases the oldest until the limit holds. */
gw_status gw_set_max_active_streams(gw_ctx *ctx, int n);

typedef struct gw_pool_stats {
    int created;           /* streams created (lazily)                    */
    int active, idle;      /* now                                          */
    int max_active;        /* the threshold                                */
    int peak_active;       /* most active at once                          */
    int pad_;
    long long ops;         /* operations issued                            */
    long long reuses;      /* operations that reused a released stream    */
    long long partial_syncs;  /* threshold reached                         */
    long long released;    /* streams released by partial synchronisation  */
    long long waited_oldest;  /* partial syncs that had to wait             */
    long long fences;      /* fences that joined pool streams             */
} gw_pool_stats;
gw_status gw_pool_stats_get(gw_ctx *ctx, gw_pool_stats *out);

/* The same policy on a host-side model, for tests and for sizing the
 * threshold: nops operations are issued one per tick of a logical clock;
 * operation i, issued at tick t, completes at tick t + duration[i]
 * (duration >= 0).  Waiting for a stream moves the clock to its completion.
 * stream_of_op[i] receives the pool stream each operation ran on (may be
 * NULL); *out the counters at the end (before any final release). */
gw_status gw_stream_pool_simulate(int max_active, int nops,
                                  const int *duration, int *stream_of_op,
                                  gw_pool_stats *out);

/* ------------------------------------------------------------------ */
/* Cannon's ring exchange (section 5, matrix multiplication): C = A B    */
/* over P ranks of one segment, BF16 operands, FP32 accumulation on the  */
/* tensor cores.                                                         */

typedef struct gw_cannon gw_cannon;

/* Segment bytes each rank needs for an N x N product over P ranks (its A
 * stripe, two B stripe buffers, its C stripe).  GW_ERR_ARG unless
 * 1 <= P <= 64 and N is a positive multiple of P. */
gw_status gw_cannon_bytes(int n, int p, size_t *per_rank);
/* A ring of P ranks (ranks 0 .. P-1 of the context's segment, which needs
 * at least P ranks of gw_cannon_bytes each).  Stripe width Ns = N / P; rank
 * r owns rows r Ns .. r Ns + Ns - 1 of A and of C.  N must be a multiple of
 * 8 (GW_ERR_ALIGN).  Needs a device context (GW_ERR_STATE). */
gw_status gw_cannon_create(gw_ctx *ctx, int n, int p, gw_cannon **out);
gw_status gw_cannon_destroy(gw_cannon *cn);
/* Load the operands: a = A and bt = B^T (that is, B in column-major order),
 * both N x N row-major arrays of BF16 bit patterns (uint16), on the host
 * (on_device = 0) or the device.  Rank r receives A's row stripe r and B's
 * column stripe r.  Synchronous. */
gw_status gw_cannon_set(gw_cannon *cn, const void *a, const void *bt,
                        int on_device);
/* The P steps of the ring, enqueued on `stream`: in step s rank r
 * multiplies its A stripe by the B column stripe it holds, writing one
 * Ns x Ns block of its C stripe, while non-blocking puts (stream pool) send
 * that stripe to rank r - 1's spare buffer; a fence orders step s + 1 after
 * them.  Runs may be repeated (the stripes keep travelling; each run writes
 * all of C).  Device waits are bounded: a kernel that gave up is reported as
 * GW_ERR_TIMEOUT by gw_cannon_sync / gw_cannon_read_c. */
gw_status gw_cannon_run(gw_cannon *cn, gw_stream stream);
/* Schedule of the block-product kernel (results are the same bits for
 * every choice; one CTA per output tile, no clusters).  tile_m: rows of a
 * CTA's 256-column output tile, 256 (default: 3 pipeline stages of 64 KB,
 * two M = 128 products per stage reading the same B tile) or 128 (4 stages
 * of 48 KB, two accumulators so a tile's epilogue overlaps the next tile's
 * products).  group: tile rows per raster group, 1 .. 1024 (default 4); the
 * CTAs running at the same time sweep a group's rows column by column.
 * GW_ERR_ARG for other values. */
gw_status gw_cannon_schedule(gw_cannon *cn, int tile_m, int group);
/* Device synchronisation and the kernel error word. */
gw_status gw_cannon_sync(gw_cannon *cn);
/* C (N x N, row-major FP32) to the host (on_device = 0) or the device,
 * after a device synchronisation. */
gw_status gw_cannon_read_c(gw_cannon *cn, void *out, int on_device);
/* Failure-detection self-test of the block-product kernel: one launch whose
 * producer issues no loads, so every wait of the MMA and epilogue warps
 * runs out after limit_us (1 us .. 2 s) and the kernel latches a timeout,
 * drains, frees its tensor memory and returns.  *expired = 1 when it did;
 * then returns GW_ERR_TIMEOUT and the context stays usable (the error word
 * is cleared). */
gw_status gw_cannon_selftest_timeout(gw_cannon *cn, unsigned limit_us, int *expired);
/* Per-launch CUDA-event timing of the block-product kernel (synchronises
 * after each launch while enabled; resets the counters). */
gw_status gw_cannon_timing(gw_cannon *cn, int enable);
gw_status gw_cannon_stats(gw_cannon *cn, double *gemm_ms, long long *launches,
                          int *grid);

/* ------------------------------------------------------------------ */
/* domains: one shot, decomposed into px*py*pz subdomains              */

/* Create a shot domain decomposed into px x py x pz subdomains (subdomain
 * (i, j, k) is rank (k*py + j)*px + i; the segment needs at least that
 * many ranks).  split_x/y/z (px/py/pz entries, may be NULL for an even
 * split, larger pieces first) give the interior extent of each slab.
 * symmetric != 0: every subdomain array is padded to the largest
 * subdomain and allocated symmetrically (offset translation); symmetric = 0:
 * exact sizes, asymmetric allocation through second-level pointers.
 * Allocates its fields from the segment; wavefields start at zero. */
gw_status gw_domain_create(gw_ctx *ctx, const gw_shot_desc *desc, int px,
                           int py, int pz, const int *split_x,
                           const int *split_y, const int *split_z,
                           int symmetric, gw_domain **out);
gw_status gw_domain_destroy(gw_domain *d);
/* Upper bound of the segment bytes a domain of this description takes
 * (symmetric px x py x pz split with even extents, nrec receivers): the
 * fields plus metadata, work items and traces.  Host only; used for
 * admission by memory budget. */
gw_status gw_domain_bytes(const gw_shot_desc *desc, int px, int py, int pz, int nrec,
                          size_t *out);
gw_status gw_domain_info_get(gw_domain *d, gw_domain_info *out);

/* Velocity model (m/s), nx*ny*nz FP64 host values.  Computes vmax on the
 * GPU, then dt (from desc.dt or desc.courant) and coef = (v dt / h)^2 in
 * FP64 on the GPU, rounded to the storage type.  Synchronises. */
gw_status gw_set_model(gw_domain *d, const double *vel_host);
/* The same from FP32 host values. */
gw_status gw_set_model_f32(gw_domain *d, const float *vel_host);
/* A z-layered model: vz[z] (m/s) for every x, y of plane z (nz values,
 * host, read during the call).  Same precompute as gw_set_model. */
gw_status gw_set_model_layered(gw_domain *d, const double *vz);

/* Ricker wavelet r(t_n) = (1 - 2 a) exp(-a), a = (pi f (n dt - 1/f))^2,
 * computed in FP64 and rounded to FP32.  Pure host function. */
gw_status gw_ricker(double f_peak, double dt, int n, float *out);

/* out_dev[i] = in_dev[i] rounded to FP32 (IEEE 754 round to nearest, ties
 * to even) on the GPU by the integer-arithmetic conversion that the FP32
 * coefficient precompute (gw_set_model_f32 into FP32 storage) uses, so that
 * a caller or a test can check it value by value.  in_dev, out_dev: n
 * elements of device memory owned by the caller.  Enqueued on `stream`,
 * no host sync; GW_ERR_ARG for NULL arrays with n > 0. */
gw_status gw_round_to_f32(const double *in_dev, float *out_dev, size_t n,
                          gw_stream stream);

/* Add a point source at global interior cell (gx, gy, gz) with wavelet
 * samples wavelet[0..n) (FP32 host; sample n is added to lap(u_n) when
 * computing u_{n+1}; steps beyond n add nothing).  Up to 16 sources.
 * Samples are kept in FP64 and rounded to the arithmetic type in the
 * kernel. */
gw_status gw_inject_source(gw_domain *d, int gx, int gy, int gz,
                           const float *wavelet, int n);
/* The same with the library's own Ricker wavelet of peak frequency f_peak
 * (Hz), sampled in FP64 at t_n = n dt with the delay 1/f_peak (the
 * formula of gw_ricker), for n < desc.nsteps.  Needs the model (dt). */
gw_status gw_inject_ricker(gw_domain *d, int gx, int gy, int gz,
                           double f_peak);
/* Receivers: nrec (x, y, z) global interior cells; trace sample n is
 * u_{n+1} at the receiver, for n < desc.nsteps.  Replaces earlier ones.
 * GW_ERR_ARG if more than 64 sources and receivers would fall inside one
 * work item (tile column of the domain's schedule); a batch whose items
 * still hold more reports GW_ERR_STATE at its next synchronisation. */
gw_status gw_set_receivers(gw_domain *d, int nrec, const int *xyz);

/* Advance nsteps steps on `stream`: K-step chunks (desc.chunk) replayed
 * from an instantiated CUDA graph, the remainder launched directly.  Each
 * step is one launch of the fused kernel over all subdomains (stencil,
 * sponge, source, receivers, norm partials and, in GW_HALO_FUSED mode, the
 * halo puts), plus the put kernel in GW_HALO_SEPARATE mode; each chunk
 * ends with the FP64 norm reduction.  Asynchronous. */
gw_status gw_step(gw_domain *d, int nsteps, gw_stream stream);
/* Refresh every subdomain's face halos of the current wavefield u_n from
 * its neighbours (pack/put/unpack kernel; Listing 1's puts). */
gw_status gw_put_halo(gw_domain *d, gw_stream stream);
/* Fence (Listing 1's ompx_fence): all puts enqueued so far are complete
 * and visible to later work on `stream`.  With sync != 0 also waits on the
 * host and reports latched device errors. */
gw_status gw_barrier(gw_domain *d, gw_stream stream, int sync);

/* Copy traces to host: out[r*nsteps + n], FP32, for r < nrec, n < nsteps
 * (<= desc.nsteps).  Synchronises the domain's work. */
gw_status gw_read_receivers(gw_domain *d, float *host_out, int nrec,
                            int nsteps);
/* Gather a field into an interior host array (FP64 if f64 != 0, else
 * FP32), unscaled.  Synchronises. */
gw_status gw_read_wavefield(gw_domain *d, int which, void *host_out,
                            int f64);
/* Scatter an interior host array (FP64 if f64 != 0, else FP32) into a
 * field, rounding to the storage type, then refresh its halos.
 * Synchronises. */
gw_status gw_write_wavefield(gw_domain *d, int which, const void *host_in,
                             int f64);
/* Per-step sum of u_{n+1}^2 (FP64 sum of FP32 partials) for steps
 * [0, n); n <= steps taken and <= desc.nsteps.  Synchronises. */
gw_status gw_norms(gw_domain *d, double *host_out, int n);
/* FP64 check reductions of the current state: norm2 = sum u_n^2 and
 * energy = sum (u_n - u_{n-1})^2 / coef - sum u_n lap(u_{n-1})
 * (conserved without source and sponge).  Either pointer may be NULL.
 * Synchronises; GW_ERR_NUMERIC if non-finite. */
gw_status gw_check(gw_domain *d, double *norm2, double *energy);

/* Allocation-free variant of gw_check, for callers that cannot allocate
 * device memory (code running while another framework holds its memory
 * pool, an embedded runtime that owns all device memory, a latency-critical
 * path that must not wait on an allocation).  The paper has no counterpart;
 * it is a library convenience.
 *
 * u_cur, u_prev, coef: device arrays of one grid in the library's padded
 * layout (element (x, y, z) at ((z + 4) * (ny + 8) + (y + 4)) * px + xoff +
 * x, xoff = 8 for GW_F32, 4 for GW_F64, 16 for GW_F16S / GW_BF16; coef is
 * FP16 for the two 16-bit types), halo cells holding the boundary values
 * (zero for a zero boundary).  px: row pitch in elements, >= xoff + nx + 4.
 * scale_u: the power-of-two scale the u arrays are stored with (1 unless
 * GW_F16S).  out_dev: 3 doubles of device memory that receive
 * sum u^2, sum (u - u_prev)^2 / coef and sum u lap(u_prev); the energy of
 * gw_check is out_dev[1] - out_dev[2].  Enqueued on `stream`, no host sync.
 *
 * The per-plane partial sums live in one built-in device array of
 * 4096 x 3 doubles (96 KiB) that every GPU which loads the library keeps
 * until the process exits: nz > 4096 is rejected with GW_ERR_ARG.  The first
 * call on a device looks up that array's device address (with the device
 * current), so make the first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (different streams, no
 * ordering between them) race; calls ordered on one stream do not.  Each
 * call overwrites the partials it uses, so nothing needs clearing.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
gw_status gw_check_fields_noalloc(const void *u_cur, const void *u_prev,
                                  const void *coef, int dtype, int nx, int ny,
                                  int nz, int px, double scale_u,
                                  double *out_dev, gw_stream stream);

/* ------------------------------------------------------------------ */
/* batches: several independent shots advanced by the same launches    */

/* Group nshots existing domains of one context (one storage type) so that
 * every launch covers the work items of all of them: shots with the same
 * kernel tile, sponge setting, address mode and halo mode share one launch
 * per step (or per chunk in persistent mode); shots that differ form
 * separate groups launched one after the other.  Shots with separate halo
 * copies (GW_HALO_SEPARATE) run one launch per step followed by their
 * halo-copy kernels, whatever `persistent` says.  Each shot keeps its own
 * model, sources, receivers, step counter and logs, read through its
 * domain.  chunk: steps per CUDA-graph chunk (0: 25; < 0: plain launches).
 * persistent != 0: one cooperative launch per group per chunk with a
 * device-wide barrier between steps, groups one after the other; otherwise
 * the groups of a chunk run side by side on streams forked from the
 * caller's and joined at the chunk's end (one graph per chunk).  The batch
 * allocates its tables from the segment; destroy it before its domains. */
gw_status gw_batch_create(gw_ctx *ctx, int nshots, gw_domain *const *shots,
                          int chunk, int persistent, gw_batch **out);
gw_status gw_batch_destroy(gw_batch *b);
/* Advance every shot of the batch by nsteps steps on `stream`. */
gw_status gw_batch_step(gw_batch *b, int nsteps, gw_stream stream);
/* Launch groups, total CTAs and work items of one step of the batch. */
gw_status gw_batch_info(gw_batch *b, int *groups, int *ctas, int *items);
/* Per-step device time of the batch's step kernels while enabled
 * (plain launches; stats as for gw_kernel_stats_get). */
gw_status gw_batch_timing(gw_batch *b, int enable);
gw_status gw_batch_stats_get(gw_batch *b, gw_kernel_stats *out);

/* Autotuner: time every kernel tile available for this storage type on a
 * scratch domain shaped like `desc` with a px x py x pz split (homogeneous
 * model, `steps` timed steps after a warm-up), using free segment memory,
 * and return the fastest tile (for gw_shot_desc.tile) and its time per
 * step.  ms_all (nullable, n_all entries) receives the time per step of
 * tile t at ms_all[t - 1] (0 for a tile that does not fit an SM).
 * Results are cached per (shape, split, storage, halo mode, sponge) for the
 * life of the context.  Synchronises. */
gw_status gw_autotune(gw_ctx *ctx, const gw_shot_desc *desc, int px, int py,
                      int pz, int steps, int *best_tile, double *best_ms,
                      double *ms_all, int n_all);
/* Tiles for a batch of n single-domain shots of one storage type: each
 * distinct shape is autotuned at full occupancy (as gw_autotune, cached, on
 * the shot's x-y plane over enough planes for 64 M points, times scaled
 * back to the shot's planes: a small shot alone would time one CTA's
 * latency rather than the tile's throughput inside a batch; the shot's own
 * shape when the segment has no room for that), then one tile
 * for every shot is chosen (the one with the least summed time) unless the
 * per-shape best tiles are faster in sum by more than `margin` (e.g. 0.05;
 * 0 when the tile groups run side by side, as a non-persistent batch's
 * do).  tiles_out[i] receives shot i's tile. */
gw_status gw_plan_tiles(gw_ctx *ctx, int n, const gw_shot_desc *descs, int steps,
                        double margin, int *tiles_out);
/* Tile model (host only, no timing): the tile expected to move the fewest
 * bytes per point for an nx x ny plane -- the staged plane's x/y halo
 * overhead plus the two pointwise fields, times the waste of partial tiles
 * at the grid edges -- among each type's main tiles.  The server uses it
 * for requests whose tile is 0. */
gw_status gw_pick_tile(int dtype, int nx, int ny, int *tile);
/* Number of kernel tiles available for a storage type (GW_F32 ...). */
gw_status gw_tile_count(int dtype, int *count);

/* ------------------------------------------------------------ serving
 * A request loop on a thread of its own: shots are submitted at any time,
 * admitted in arrival order while their footprint (gw_domain_bytes) fits
 * the HBM budget and a slot is free, kept resident, and advanced together
 * in multi-shot batches (one per storage type) whose membership changes at
 * chunk boundaries: a shot that arrives while others run joins the next
 * chunk, a finished shot leaves it.  A chunk never runs past the end of a
 * member shot, so each shot takes exactly its own steps and its results
 * are those of the same shot run alone.  The segment of `ctx` must hold
 * the budget plus the batch tables; the caller keeps it attached for the
 * server's life. */
typedef struct gw_server gw_server;

typedef struct gw_request {
    gw_shot_desc desc;     /* one single-domain shot of desc.nsteps steps  */
    const float *vel;      /* nz*ny*nx host velocities (m/s), read when the
                              shot is admitted: the caller keeps it valid
                              until the ticket completes; or NULL and vz  */
    const double *vz;      /* nz velocities of a z-layered model; copied
                              by gw_submit                                 */
    int src[3];            /* Ricker source cell (x, y, z)                 */
    double f_peak;         /* Ricker peak frequency, Hz                    */
    int nrec;              /* receivers, nrec x (x, y, z) in rec, copied   */
    const int *rec;
    float *traces;         /* host [nrec][nsteps], written before the
                              ticket completes; NULL: not returned         */
} gw_request;

typedef struct gw_result {
    int status;            /* GW_OK or the error that ended the shot       */
    int steps;
    long long points;      /* interior points                              */
    double submit_s;       /* server clock (s since gw_server_create)      */
    double admit_s;
    double done_s;         /* traces on the host                           */
    double norm2;          /* gw_check of the final state                  */
    double energy;
    size_t device_bytes;   /* footprint charged against the budget         */
    int tile;
} gw_result;

typedef struct gw_server_stats {
    int pending, active, completed, max_active;
    int chunks;            /* chunk launches so far                        */
    int rebuilds;          /* batch rebuilds (membership changes)          */
    size_t budget_bytes, used_bytes, peak_bytes;
    long long point_updates;
    double busy_s;         /* time with at least one shot active           */
    double now_s;          /* server clock                                 */
} gw_server_stats;

/* max_slots: most shots resident at once; chunk: steps per batch chunk
 * (0: 25).  The server runs each storage type on a non-blocking stream of its own. */
gw_status gw_server_create(gw_ctx *ctx, size_t hbm_budget, int max_slots, int chunk,
                           gw_server **out);
/* Stops the loop after the running chunk; shots not finished end with
 * GW_ERR_STATE. */
gw_status gw_server_destroy(gw_server *s);
/* GW_ERR_BUDGET if the shot's footprint exceeds the whole budget. */
gw_status gw_submit(gw_server *s, const gw_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: forever) for a ticket; GW_ERR_TIMEOUT if it
 * has not completed.  A completed ticket is returned once. */
gw_status gw_wait(gw_server *s, uint64_t ticket, int timeout_ms, gw_result *out);
gw_status gw_server_stats_get(gw_server *s, gw_server_stats *out);
/* Server clock in seconds (the clock of gw_result). */
double gw_server_now(gw_server *s);

/* Failure-detection self-test: one warp waits on an mbarrier nobody
 * arrives on and on a device counter nobody increments -- the two kinds of
 * wait of the step kernel -- each bounded by limit_us (1 us .. 2 s; the
 * step kernel bounds them by 4 s).  *expired receives one bit per wait that
 * gave up (1: mbarrier, 2: counter).  Returns GW_ERR_TIMEOUT when a wait
 * gave up (the expected outcome); the context stays usable.  Synchronises
 * the legacy stream. */
gw_status gw_selftest_timeout(gw_ctx *ctx, unsigned limit_us, int *expired);

/* Record the device time of every step-kernel launch (CUDA events) while
 * enabled; gw_kernel_stats_get returns the totals and resets them. */
gw_status gw_kernel_timing(gw_domain *d, int enable);
gw_status gw_kernel_stats_get(gw_domain *d, gw_kernel_stats *out);

/* Raw storage copy of the whole state (both wavefields, step counter) for
 * checkpoint/restart; gw_state_bytes gives the size.  Synchronises. */
gw_status gw_state_bytes(gw_domain *d, size_t *bytes);
gw_status gw_save_state(gw_domain *d, void *host_out);
gw_status gw_load_state(gw_domain *d, const void *host_in);

#ifdef __cplusplus
}
#endif
#endif /* GBWAVE_H */
