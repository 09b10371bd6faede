// gw_device.h -- plain-old-data structures shared by the host runtime and
// the sm_103a kernels of the Minimod acoustic-isotropic step.
//
// Memory layout of one subdomain field ("padded array"): interior point
// (x, y, z) of an nx x ny x nz subdomain lives at element
//     ((z + R) * py + (y + R)) * px + (x + xoff)
// with R = 4 halo cells in y and z, a halo of xoff >= R cells in x chosen
// so that the interior x origin is 32-byte (sector) aligned (xoff = 8 for
// FP32, 4 for FP64, 16 for 16-bit storage), py = ny + 2R rows per plane and
// the row pitch px a multiple of 32 bytes.  The array holds nz + 2R planes.
// Halo cells of a subdomain are written only by halo puts (or stay zero at
// a non-periodic global boundary); padding beyond x = nx + R is never
// written and stays zero.
#pragma once
#include <stdint.h>

namespace gw {

constexpr int R = 4;               // stencil radius (8th order)
constexpr int kMaxSources = 16;    // point sources per shot
constexpr int kMaxLocal = 64;      // receivers/sources inside one work item
constexpr int kMapsPerSub = 6;     // tensor maps per subdomain

// tensor-map slots per subdomain
enum MapSlot {
    MAP_U0_HALO = 0,   // u buffer 0, box (TX + 2 xoff) x (TY + 2R) x 1
    MAP_U1_HALO = 1,   // u buffer 1, same box
    MAP_U0_PW = 2,     // u buffer 0, box TX x TY x 1 (pointwise)
    MAP_U1_PW = 3,     // u buffer 1, pointwise
    MAP_COEF_PW = 4,   // coefficient field, pointwise
    MAP_W_PW = 5       // w field (delta storage), pointwise
};

// error bits latched by kernels in the device error word
enum ErrBits : unsigned {
    ERRB_TIMEOUT = 1u,      // a bounded mbarrier / grid-barrier wait gave up
    ERRB_NONFINITE = 2u,    // a norm reduction saw inf/nan
    ERRB_LOCAL_OVERFLOW = 4u,  // too many receivers/sources in one item
    ERRB_BAD_ITEM = 8u      // a work item failed its bounds check
};

struct SubDev {
    char *u[2];            // the two wavefield buffers (ping-pong)
    char *w;               // delta storage: w_n (nullptr otherwise)
    char *coef;            // coefficient field
    int nx, ny, nz;        // interior extents
    int gx0, gy0, gz0;     // global origin of the interior
    int px, py;            // row pitch (elements), rows per plane
    int shot;              // owning shot
    int rank;              // rank (segment slot) of this subdomain
    int nbr[6];            // subdomain index across -x,+x,-y,+y,-z,+z (-1)
    int pad_[2];
};

struct ShotDev {
    int *step;             // device step counter n (steps taken)
    const double *wavelet; // [nsrc][cap] source samples
    float *traces;         // [nrec][cap]
    double *norms;         // [cap] per-step sum of u_{n+1}^2
    const double *gx, *gy, *gz;  // global sponge profiles (rounded to the
                                 // math type when loaded)
    const int4 *src;       // nsrc (x, y, z, 0) global cells
    const int4 *rec;       // nrec (x, y, z, 0) global cells
    int cap;               // capacity of wavelet / traces / norms
    int nsrc, nrec;
    int NX, NY, NZ;        // global interior extents
    int first_item, nitems;   // this shot's work items (contiguous range)
    float su, sw;          // delta storage scales (powers of two)
    float isu, isw;        // their inverses
    int lo[2][3], hi[2][3];   // bounding boxes of the sources [0] and of the
                              // receivers [1] (global cells; lo > hi: none)
    int limit;             // steps the shot takes at most: launches skip its
                           // items from step `limit` on and its counter
                           // stops there (INT_MAX: no limit)
};

// One work item: a tile column (x0, y0) of subdomain `sub`, planes [z0, z1).
struct Item {
    int sub;
    int xy;                // x0 | (y0 << 16)
    int z0, z1;
};

// Kernel arguments, passed by value as a __grid_constant__ parameter.
struct StepArgs {
    const SubDev *subs;
    const ShotDev *shots;
    const Item *items;
    const void *maps;      // CUtensorMap[nsub][kMapsPerSub], 64-B aligned
    double *partials;      // [chunk][nitems] FP64 norm partials
    unsigned *err;         // device error word
    char *seg_base;        // segment base (symmetric address translation)
    long long rank_stride; // bytes between rank segments
    int nitems;
    int k;                 // step index within the chunk of the first step
    int nk;                // steps this launch performs (persistent: > 1)
    unsigned *gbar;        // device-wide barrier counter (zero at launch)
    unsigned *ctr;         // work-item tickets (zero between steps; the
                           // kernel resets it after each step)
    int dynamic;           // 1: CTAs take items from ctr; 0: b, b + grid, ...
    int symmetric;         // 1: neighbour address = own + (dr * stride)
    int fused_halo;        // 1: epilogue stores into neighbours' halos
};

}  // namespace gw
