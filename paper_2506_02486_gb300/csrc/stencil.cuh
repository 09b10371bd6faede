// stencil.cuh -- the fused Minimod acoustic-isotropic step for sm_103a.
//
// One launch advances every subdomain of every shot in the launch by one
// leapfrog step (8th-order 25-point star Laplacian, Cerjan sponge, point
// sources, receivers, FP64 norm partials, and -- in fused-halo mode -- the
// one-sided puts of the new boundary planes into the neighbours' halos,
// the device-side form of Listing 1's ompx_put; the paper's section 4.5).
//
// Work decomposition.  A work item is a tile column: TX x TY points of one
// subdomain over planes [z0, z1).  Items are ordered z-chunk-major so that
// the CTAs running at the same time hold neighbouring columns at the same
// depth (their x/y halo strips are then served from L2), and CTA b takes
// items b, b + grid, b + 2 grid, ...
//
// Warp specialisation.  Each CTA has NT/32 consumer warps and one producer
// warp.  The producer streams, in consumption order and across item
// boundaries, two rings of shared-memory slots filled by TMA
// (cp.async.bulk.tensor, completion counted on "full" mbarriers):
//   * the u ring (SU slots): plane p of u_n with its x/y halo, box
//     (TX + 2 xoff) x (TY + 8);
//   * the pointwise ring (SP slots): the TX x TY tiles of the second state
//     field (u_{n-1}, or w_n for delta storage) and of coef at plane z.
// Consumers hand slots back warp by warp through "empty" mbarriers, so no
// CTA-wide barrier sits in the z loop.  Each consumer thread owns 4
// consecutive x points (one 128-bit group for FP32) of PY rows.  Its z
// neighbours come from a 9-deep register queue filled from the plane that
// just arrived; x/y neighbours come from the staged plane.
//
// Arithmetic order (fixed, so that decomposed and undecomposed runs and
// mirror-image points give identical bits):
//   s_m = ((u[x-m] + u[x+m]) + (u[y-m] + u[y+m])) + (u[z-m] + u[z+m])
//   lap = fma(c4, s4, fma(c3, s3, fma(c2, s2, fma(c1, s1, (3 c0) u))))
//   lap += wavelet[n] at a source cell
//   3-level: u' = G * fma(coef, lap, fma(-G, u_prev, u + u))
//   delta:   w' = G * fma(coef, lap, w);  u' = fma(G, u, w')
// with G = (g_x g_y) g_z from per-axis tables on global coordinates.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "gw_device.h"
#include "gw_kernels.h"
#include "ptx.cuh"

namespace gw {

// ---------------------------------------------------------------- storage

template <class T> struct St;

// XO: x offset of the interior in a padded global row (32-byte aligned, so
// rows of a tile are written and read in whole sectors); HL: x halo staged
// in shared memory (>= R and a multiple of 16 bytes, a TMA requirement on
// the box's first coordinate).
template <> struct St<float> {
    using M = float;
    static constexpr int XO = 8, HL = 4;
    __device__ __forceinline__ static void ld4(const float *p, M v[4])
    {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    // u_{n+1} is read again only in the next step, after the whole grid has
    // passed through L2: stored with the evict-first (streaming) hint so
    // that it does not push out the u_n planes whose x/y halo strips the
    // neighbouring tiles still read (512^3: 1.0-1.5 % faster)
    __device__ __forceinline__ static void st4(float *p, const M v[4])
    {
        asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};"
                     :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]) : "memory");
    }
    __device__ __forceinline__ static void st1(float *p, M v) { *p = v; }
};

template <> struct St<double> {
    using M = double;
    static constexpr int XO = 4, HL = 4;
    __device__ __forceinline__ static void ld4(const double *p, M v[4])
    {
        double2 a = reinterpret_cast<const double2 *>(p)[0];
        double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ static void st4(double *p, const M v[4])
    {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
    __device__ __forceinline__ static void st1(double *p, M v) { *p = v; }
};

template <> struct St<__half> {
    using M = float;
    static constexpr int XO = 16, HL = 8;
    __device__ __forceinline__ static void ld4(const __half *p, M v[4])
    {
        uint2 q = *reinterpret_cast<const uint2 *>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&q.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ static void st4(__half *p, const M v[4])
    {
        __half2 a = __floats2half2_rn(v[0], v[1]);
        __half2 b = __floats2half2_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t *>(&a);
        q.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    __device__ __forceinline__ static void st1(__half *p, M v) { *p = __float2half_rn(v); }
};

template <> struct St<__nv_bfloat16> {
    using M = float;
    static constexpr int XO = 16, HL = 8;
    __device__ __forceinline__ static void ld4(const __nv_bfloat16 *p, M v[4])
    {
        uint2 q = *reinterpret_cast<const uint2 *>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&q.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ static void st4(__nv_bfloat16 *p, const M v[4])
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t *>(&a);
        q.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = q;
    }
    __device__ __forceinline__ static void st1(__nv_bfloat16 *p, M v)
    {
        *p = __float2bfloat16_rn(v);
    }
};

// Rounded-once arithmetic in the math type (no contraction by the compiler).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// 8th-order central second-difference weights (Taylor table), with the
// centre weight already multiplied by 3 for the three axes.
template <class M> struct W {
    static constexpr M c0x3 = M(-615.0 / 72.0);
    static constexpr M c1 = M(8.0 / 5.0);
    static constexpr M c2 = M(-1.0 / 5.0);
    static constexpr M c3 = M(8.0 / 315.0);
    static constexpr M c4 = M(-1.0 / 560.0);
};

// ---------------------------------------------------------------- config

template <class T_, int TX_, int TY_, int PY_, int SU_, int SP_,
          int MINB_ = 1, bool PACK_ = true, int KP_ = 2>
struct Cfg {
    using T = T_;
    using M = typename St<T>::M;
    // coefficient storage: FP16 next to 16-bit wavefields, else T
    using CT = typename std::conditional<sizeof(T_) == 2, __half, T_>::type;
    static constexpr int TX = TX_, TY = TY_, PY = PY_, SU = SU_, SP = SP_;
    static constexpr int NTX = TX / 4, NTY = TY / PY, NT = NTX * NTY;
    static constexpr int NCW = NT / 32;              // consumer warps
    static constexpr int THREADS = NT + 32;          // + one producer warp
    // registers per thread: each of the SM's 4 sub-partitions owns 16K
    // registers and hosts ceil(warps / 4) of this CTA's warps
    static constexpr int MINB = MINB_;               // CTAs per SM wanted
    static constexpr bool PACK = PACK_;              // f32x2 arithmetic
    static constexpr int KP = KP_;                   // planes per queue shift
    static constexpr int WPP = (THREADS / 32 + 3) / 4;
    static constexpr int MAXREG_ = (16384 / (WPP * MINB * 32)) / 8 * 8;
    static constexpr int MAXREG = MAXREG_ > 255 ? 255 : MAXREG_;
    static constexpr int XO = St<T>::XO;
    static constexpr int HL = St<T>::HL;
    static constexpr int RW = TX + 2 * HL;          // smem row (elements)
    static constexpr int UROWS = TY + 2 * R;
    static constexpr int UBYTES = RW * UROWS * (int)sizeof(T);
    static constexpr int PBYTES = TX * TY * (int)sizeof(T);
    // slot strides padded to the 128-byte alignment of TMA destinations
    static constexpr int USTRIDE = (UBYTES + 127) / 128 * 128;
    static constexpr int PSTRIDE = (PBYTES + 127) / 128 * 128;
    static constexpr int OFF_P = SU * USTRIDE;
    static constexpr int OFF_BAR = OFF_P + SP * 2 * PSTRIDE;
    static constexpr int OFF_LOC = OFF_BAR + 16 * (SU + SP);   // full + empty
    static constexpr int OFF_MISC = OFF_LOC + 16 * kMaxLocal;
    static constexpr int OFF_RED = OFF_MISC + 16;
    static constexpr int OFF_NBR = OFF_RED + 8 * NCW;     // 6 x NbrPut (32 B)
    // work-item ring from the producer to the consumers: IQ item indices,
    // then IQ full and IQ empty mbarriers
    static constexpr int IQ = 4;
    static constexpr int OFF_IQ = OFF_NBR + 32 * 6;
    static constexpr int SMEM = OFF_IQ + 4 * IQ + 16 * IQ;
    static_assert(TX % 4 == 0 && TY % PY == 0 && NT % 32 == 0, "tile");
    static_assert((RW * (int)sizeof(T)) % 16 == 0, "TMA box row");
    static_assert(SU >= 6 && SP >= 2, "ring depth");
};

// Bounded wait that also gives up at once when another thread of the CTA
// already gave up (shared abort flag): a timed-out CTA drains quickly.
__device__ __forceinline__ bool wait_slot(uint64_t *bar, uint32_t parity,
                                          volatile int *abortf)
{
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = global_timer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0) {
            if (*abortf) return false;
            if (global_timer() - t0 > kWaitLimitNs) return false;
        }
    }
}

// Barrier among the consumer warps only (the producer warp is not part).
__device__ __forceinline__ void consumer_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" :: "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------- groups

// Four consecutive x points of one row.  For packed FP32 arithmetic they
// are held as two float2 pairs, so packed operands are always aligned
// register pairs and never need moving; otherwise as four scalars.
template <class M, bool P> struct Grp {
    M v[4];
    __device__ __forceinline__ M get(int i) const { return v[i]; }
    __device__ __forceinline__ void set(int i, M x) { v[i] = x; }
};
template <> struct Grp<float, true> {
    float2 a, b;
    __device__ __forceinline__ float get(int i) const
    {
        return i == 0 ? a.x : i == 1 ? a.y : i == 2 ? b.x : b.y;
    }
    __device__ __forceinline__ void set(int i, float x)
    {
        if (i == 0) a.x = x; else if (i == 1) a.y = x; else if (i == 2) b.x = x; else b.y = x;
    }
    __device__ __forceinline__ float2 pair(int h) const { return h ? b : a; }
};

// Load a group of storage type T from shared memory.
template <class T, bool P>
__device__ __forceinline__ void ld_grp(const T *p, Grp<typename St<T>::M, P> &g)
{
    typename St<T>::M v[4];
    St<T>::ld4(p, v);
#pragma unroll
    for (int i = 0; i < 4; ++i) g.set(i, v[i]);
}
template <>
__device__ __forceinline__ void ld_grp<float, true>(const float *p, Grp<float, true> &g)
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    g.a = make_float2(q.x, q.y);
    g.b = make_float2(q.z, q.w);
}
template <>
__device__ __forceinline__ void ld_grp<__half, true>(const __half *p, Grp<float, true> &g)
{
    uint2 q = *reinterpret_cast<const uint2 *>(p);
    g.a = __half22float2(*reinterpret_cast<__half2 *>(&q.x));
    g.b = __half22float2(*reinterpret_cast<__half2 *>(&q.y));
}
template <>
__device__ __forceinline__ void ld_grp<__nv_bfloat16, true>(const __nv_bfloat16 *p,
                                                           Grp<float, true> &g)
{
    uint2 q = *reinterpret_cast<const uint2 *>(p);
    g.a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&q.x));
    g.b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&q.y));
}

// ---------------------------------------------------------------- kernel

// Where the fused halo puts of the current item go, per face: the
// neighbour's buffer receiving u_{n+1} and its strides, resolved once per
// item (symmetric: own buffer + rank distance x rank stride; asymmetric: the
// resolved second-level pointer) and kept in shared memory.
struct NbrPut {
    char *base;            // neighbour's u_{n+1} buffer (nullptr: no neighbour)
    long long plane;       // elements per plane
    int px;                // row pitch (elements)
    int ext;               // neighbour extent along the face normal
    int pad_[2];
};
static_assert(sizeof(NbrPut) == 32, "NbrPut size");

template <class C, bool DELTA, bool SPONGE>
struct Step {
    using T = typename C::T;
    using M = typename C::M;
    using S = St<T>;
    static constexpr int TX = C::TX, TY = C::TY, PY = C::PY;
    static constexpr int SU = C::SU, SP = C::SP, XO = C::XO, HL = C::HL;

    const StepArgs &A;
    unsigned char *smem;
    int tid, tx, ty, lane;

    // consumer
    unsigned tg, jg;           // u loads / pointwise planes consumed
    // their ring positions, kept as running counters (the ring depths need
    // not be powers of two, and a division per use costs instructions in
    // the loop): tg % SU and (tg / SU) & 1, (tg - R) % SU, jg % SP and
    // (jg / SP) & 1
    unsigned us, uph, cs, pss, pph;
    unsigned itn_;             // work items taken from the ring
    int kk;                    // step index within the chunk being computed
    bool aborted;              // a wait of this thread gave up

    // current item (cached in registers: the stores below may alias the
    // global tables, so nothing is re-read from them inside the z loop)
    int sub, x0, y0, z0, z1, n, par;
    int nx, ny, nz;
    int vx;                    // valid x points of this thread (0..4)
    bool rowok[PY];
    int px_;                   // row pitch (elements)
    size_t plane_;             // plane stride (elements)
    int nbr_[6];
    int rank_;
    int nl_;                   // receivers + sources inside this item
    bool item_puts;            // fused puts: this tile touches a face with a neighbour
    bool fast_;                // whole tile
    int zloc_lo_, zloc_hi_;    // planes holding this item's sources / receivers
    T *ust;                    // store address of this thread's first row at the compute plane
    long long wdelta;          // w field minus u_{n+1} field (elements)
    size_t roff_[PY];          // in-plane element offset of each row's first point
    M isu_, q_, iq_;           // 1/su; q = sw/su and su/sw (delta storage)
    // FP16 delta storage carries power-of-two scales; BF16 does not
    static constexpr bool SCALED = DELTA && std::is_same<T, __half>::value;
    const double *gz_ptr;      // sponge factors along z of this subdomain
    M gz_next;                 // sponge factor of the next plane (prefetched)
    int cap_;
    const SubDev *sd;
    const ShotDev *sh;
    T *unext, *wbuf;
    // packed FP32 arithmetic on float2 pairs (Blackwell f32x2 add/mul/fma)
    static constexpr bool PK = std::is_same<M, float>::value && C::PACK;
    using G = Grp<M, PK>;
    // planes per trip of the z loop: the register queue shifts by KP planes
    // once per trip (KP planes of phases share one shift)
    static constexpr int KP = C::KP;
    static_assert(KP == 2 || KP == 4, "planes per trip");
    G gxy[PY];                 // g_x g_y of this thread's points
    // sum of u'^2: a thread's (at most 4 PY = 8) points of one plane are
    // summed in the math type; the plane sums are accumulated as an
    // unevaluated pair (nacc + ncomp) by error-free transformations (TwoSum,
    // the cascaded summation "Sum2" of Ogita, Rump and Oishi, 2005), which
    // is as accurate as an FP64 accumulator, and the pair is added in FP64
    // at the end of the item.  (An FP64 add per plane stalls every warp on
    // GB300's narrow FP64 pipe: -1 % FP32, -9 % 16-bit storage at 512^3.)
    M nacc, ncomp;
    G Q[8 + KP][PY];           // this thread's points on planes z-4 .. z+4+KP-1

    __device__ Step(const StepArgs &a, unsigned char *sm) : A(a), smem(sm) {}

    __device__ T *ubuf(unsigned slot)
    {
        return reinterpret_cast<T *>(smem + slot * C::USTRIDE);
    }
    __device__ T *pbuf(unsigned slot, int f)
    {
        return reinterpret_cast<T *>(smem + C::OFF_P +
                                     (slot * 2 + f) * C::PSTRIDE);
    }
    __device__ uint64_t *bars() { return reinterpret_cast<uint64_t *>(smem + C::OFF_BAR); }
    __device__ uint64_t *ufull(unsigned s) { return bars() + s; }
    __device__ uint64_t *pfull(unsigned s) { return bars() + SU + s; }
    __device__ uint64_t *uempty(unsigned s) { return bars() + SU + SP + s; }
    __device__ uint64_t *pempty(unsigned s) { return bars() + 2 * SU + SP + s; }
    __device__ int4 *loc() { return reinterpret_cast<int4 *>(smem + C::OFF_LOC); }
    __device__ int *misc() { return reinterpret_cast<int *>(smem + C::OFF_MISC); }
    __device__ volatile int *abortf() { return misc() + 1; }
    __device__ double *red() { return reinterpret_cast<double *>(smem + C::OFF_RED); }
    __device__ NbrPut *nbrput() { return reinterpret_cast<NbrPut *>(smem + C::OFF_NBR); }
    __device__ volatile int *itemq() { return reinterpret_cast<volatile int *>(smem + C::OFF_IQ); }
    __device__ uint64_t *iqfull(unsigned s)
    {
        return reinterpret_cast<uint64_t *>(smem + C::OFF_IQ + 4 * C::IQ) + s;
    }
    __device__ uint64_t *iqempty(unsigned s) { return iqfull(0) + C::IQ + s; }

    // ---- work items ---------------------------------------------------
    // Static schedule (A.dynamic == 0): CTA b takes items b, b + grid, ....
    // Dynamic schedule: the CTAs take a step's items in order from a ticket
    // counter (A.ctr, zero at the start of every step); every CTA draws
    // tickets until it gets one past the last item, so a step hands out
    // exactly nitems + gridDim.x tickets, and the CTA that draws the last
    // one resets the counter for the next step.  A CTA held up by a costly
    // item (a partial tile, halo puts, sources) takes fewer, and the CTAs
    // running at the same time stay on neighbouring tiles.  Either way the
    // producer claims the items (it streams ahead) and hands their indices
    // to the consumers through a ring of IQ slots.
    __device__ __forceinline__ int claim_item(unsigned &nth)
    {
        if (!A.dynamic) {
            const unsigned t = blockIdx.x + gridDim.x * nth++;
            if (t < (unsigned)A.nitems) return (int)t;
            nth = 0;
            return -1;
        }
        const unsigned t = atomicAdd(A.ctr, 1u);
        if (t == (unsigned)A.nitems + gridDim.x - 1u) atomicExch(A.ctr, 0u);
        return t < (unsigned)A.nitems ? (int)t : -1;
    }

    // producer: item index (-1: none left in this step) into slot q % IQ
    __device__ __forceinline__ bool publish_item(int v, unsigned &q)
    {
        const unsigned s = q % C::IQ;
        if (q >= (unsigned)C::IQ && !wait_slot(iqempty(s), ((q / C::IQ) - 1) & 1u, abortf()))
            return false;
        itemq()[s] = v;
        mbar_arrive(iqfull(s));       // release: the index is visible to the waiter
        ++q;
        return true;
    }

    // consumers: the next item of this step, the same value in every
    // consumer thread (-1: the step is done; -2: this CTA gave up).  One
    // thread takes it from the ring and the consumer barrier broadcasts it,
    // so that all consumer threads always take the same path.
    __device__ __forceinline__ int next_item()
    {
        if (tid == 0) {
            const unsigned s = itn_ % C::IQ;
            int v = -2;
            if (wait_slot(iqfull(s), (itn_ / C::IQ) & 1u, abortf())) {
                v = itemq()[s];
                mbar_arrive(iqempty(s));
            }
            misc()[2] = v;
        }
        ++itn_;
        consumer_sync(C::NT);
        return misc()[2];
    }


    __device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity)
    {
        // a completed phase needs no more than one probe; the bounded loop
        // (and the abort bookkeeping) is the slow path
        if (mbar_try_wait(bar, parity)) return true;
        if (aborted) return false;
        if (!wait_slot(bar, parity, abortf())) {
            if (!*abortf()) atomicOr(A.err, ERRB_TIMEOUT);
            *abortf() = 1;
            aborted = true;
            return false;
        }
        return true;
    }

    // ---- producer warp (one lane) ------------------------------------
    __device__ void produce()
    {
        // Normal L2 priority for the pointwise stream: marking it evict-first
        // cost ~6 % at 512^3 (u_{n-1} is overwritten in place by the same
        // CTA a few microseconds after it is read).  FP32 u planes are kept
        // with priority (evict-last) for the neighbouring tiles' halo reads
        // (with the streaming stores: 512^3 1.0-1.5 %, 1200^3 0.6 % faster;
        // the 16-bit tiles gained nothing from either hint).
        const uint64_t pol_u = std::is_same<T, float>::value ? policy_evict_last()
                                                            : policy_evict_normal();
        const uint64_t pol_p = policy_evict_normal();
        unsigned L = 0, P = 0, iqn = 0, nth = 0;
        for (int k = 0; k < A.nk; ++k) {
        if (k > 0) {
            // the previous step's stores must be complete everywhere before
            // this CTA streams the planes of the next one
            if (!wait_count(A.gbar, (unsigned)k * gridDim.x, abortf())) {
                if (!*abortf()) atomicOr(A.err, ERRB_TIMEOUT);
                *abortf() = 1;
                goto drain;
            }
            fence_proxy_async_global();
        }
        for (;;) {
            const int it = claim_item(nth);
            Item I{};
            int n = 0;
            if (it >= 0) {
                I = A.items[it];
                const ShotDev &sh0 = A.shots[A.subs[I.sub].shot];
                n = *sh0.step + A.k + k;
                // a shot that has taken all its steps (a batch member that
                // finishes inside the chunk) is left as it is
                if (n >= sh0.limit) continue;
            }
            if (!publish_item(it, iqn)) {
                *abortf() = 1;
                goto drain;
            }
            if (it < 0) break;
            const int p = n & 1;
            const char *base = static_cast<const char *>(A.maps) +
                               (size_t)I.sub * kMapsPerSub * 128;
            const char *map_u = base + (p ? MAP_U1_HALO : MAP_U0_HALO) * 128;
            const char *map_a = base + (DELTA ? MAP_W_PW : (p ? MAP_U0_PW : MAP_U1_PW)) * 128;
            const char *map_b = base + MAP_COEF_PW * 128;
            tensormap_acquire(map_u);
            tensormap_acquire(map_a);
            tensormap_acquire(map_b);
            // padded coordinates of the boxes: interior (x0 - HL, y0 - R)
            // for the halo box, (x0, y0) for the pointwise tiles
            const int ux = (I.xy & 0xffff) + XO - HL, uy = I.xy >> 16;
            const int T = I.z1 - I.z0 + 2 * R;
            for (int t = 0; t < T; ++t) {
                unsigned slot = L % SU;
                if (L >= SU && !wait_slot(uempty(slot), ((L / SU) - 1) & 1u, abortf())) {
                    *abortf() = 1;
                    goto drain;
                }
                mbar_arrive_expect_tx(ufull(slot), C::UBYTES);
                tma_load_3d(ubuf(slot), map_u, ufull(slot), ux, uy, I.z0 + t, pol_u);
                ++L;
                if (t >= 2 * R) {
                    unsigned ps = P % SP;
                    if (P >= SP && !wait_slot(pempty(ps), ((P / SP) - 1) & 1u, abortf())) {
                        *abortf() = 1;
                        goto drain;
                    }
                    mbar_arrive_expect_tx(pfull(ps), 2 * C::PBYTES);
                    const int zz = I.z0 + t - R;   // padded z of interior z
                    tma_load_3d(pbuf(ps, 0), map_a, pfull(ps), ux + HL, uy + R, zz, pol_p);
                    tma_load_3d(pbuf(ps, 1), map_b, pfull(ps), ux + HL, uy + R, zz, pol_p);
                    ++P;
                }
            }
        }
        }
    drain:
        // leave only after every copy issued into this CTA's shared memory
        // has landed (bounded)
        for (unsigned q = L > SU ? L - SU : 0; q < L; ++q)
            if (!wait_slot(ufull(q % SU), (q / SU) & 1u, abortf())) break;
        for (unsigned q = P > SP ? P - SP : 0; q < P; ++q)
            if (!wait_slot(pfull(q % SP), (q / SP) & 1u, abortf())) break;
    }

    // ---- item set-up ----------------------------------------------------
    __device__ __forceinline__ void begin_item(int it)
    {
        Item I = A.items[it];
        sub = I.sub;
        sd = &A.subs[sub];
        sh = &A.shots[sd->shot];
        x0 = I.xy & 0xffff;
        y0 = I.xy >> 16;
        z0 = I.z0;
        z1 = I.z1;
        nx = sd->nx; ny = sd->ny; nz = sd->nz;
        px_ = sd->px;
        plane_ = (size_t)sd->px * sd->py;
        rank_ = sd->rank;
#pragma unroll
        for (int f = 0; f < 6; ++f) nbr_[f] = sd->nbr[f];
        isu_ = (M)sh->isu;
        q_ = (M)(sh->sw * sh->isu);
        iq_ = (M)(sh->su * sh->isw);
        cap_ = sh->cap;
        gz_ptr = sh->gz + sd->gz0;
        if (SPONGE) gz_next = (M)__ldg(gz_ptr + z0);
        n = *sh->step + kk;
        par = n & 1;
        unext = reinterpret_cast<T *>(sd->u[par ^ 1]);
        wbuf = reinterpret_cast<T *>(sd->w);
        int xs = x0 + 4 * tx;
        vx = min(4, max(0, nx - xs));
#pragma unroll
        for (int r = 0; r < PY; ++r) {
            rowok[r] = (y0 + PY * ty + r) < ny;
            roff_[r] = (size_t)(y0 + PY * ty + r + R) * px_ + XO + xs;
        }
        item_puts = A.fused_halo &&
                    ((x0 < R && nbr_[0] >= 0) || (x0 + TX > nx - R && nbr_[1] >= 0) ||
                     (y0 < R && nbr_[2] >= 0) || (y0 + TY > ny - R && nbr_[3] >= 0) ||
                     (z0 < R && nbr_[4] >= 0) || (z1 > nz - R && nbr_[5] >= 0));
        if (SPONGE) {
#pragma unroll
            for (int r = 0; r < PY; ++r) {
                int gy = min(sd->gy0 + y0 + PY * ty + r, sh->NY - 1);
                M fy = (M)__ldg(sh->gy + gy);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int gx = min(sd->gx0 + xs + i, sh->NX - 1);
                    gxy[r].set(i, mul_rn((M)__ldg(sh->gx + gx), fy));
                }
            }
        }
        nacc = M(0);
        ncomp = M(0);
        // receivers and sources inside this item -> shared list (warp 0)
        if (tid < 32) {
            int cnt = 0;
            int gxa = sd->gx0 + x0, gya = sd->gy0 + y0, gza = sd->gz0;
            int xl_end = min(TX, nx - x0), yl_end = min(TY, ny - y0);
            for (int pass = 0; pass < 2; ++pass) {
                // only items that meet the box of the list search it
                const int *lo = sh->lo[pass], *hi = sh->hi[pass];
                if (!(gxa <= hi[0] && gxa + xl_end - 1 >= lo[0] &&
                      gya <= hi[1] && gya + yl_end - 1 >= lo[1] &&
                      gza + z0 <= hi[2] && gza + z1 - 1 >= lo[2]))
                    continue;
                int nlist = pass == 0 ? sh->nsrc : sh->nrec;
                const int4 *list = pass == 0 ? sh->src : sh->rec;
                for (int b = 0; b < nlist; b += 32) {
                    int e = b + lane;
                    bool in = false;
                    int4 q = make_int4(0, 0, 0, 0);
                    if (e < nlist) {
                        int4 g = list[e];
                        int lx = g.x - gxa, ly = g.y - gya, lz = g.z - gza;
                        in = lx >= 0 && lx < xl_end && ly >= 0 && ly < yl_end &&
                             lz >= z0 && lz < z1;
                        q = make_int4(pass == 0 ? -1 - e : e, lx | (ly << 16), lz, 0);
                    }
                    unsigned m = __ballot_sync(0xffffffffu, in);
                    int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (in) {
                        if (pos < kMaxLocal) loc()[pos] = q;
                        else atomicOr(A.err, ERRB_LOCAL_OVERFLOW);
                    }
                    cnt += __popc(m);
                }
            }
            if (lane == 0) misc()[0] = min(cnt, kMaxLocal);
        }
        if (tid == 32 && item_puts) {
            for (int f = 0; f < 6; ++f) {
                NbrPut q{};
                const int nb = nbr_[f];
                if (nb >= 0) {
                    const SubDev &o = A.subs[nb];
                    q.base = A.symmetric
                                 ? reinterpret_cast<char *>(unext) +
                                       (long long)(o.rank - rank_) * A.rank_stride
                                 : o.u[par ^ 1];
                    q.plane = (long long)o.px * o.py;
                    q.px = o.px;
                    q.ext = (f >> 1) == 0 ? o.nx : (f >> 1) == 1 ? o.ny : o.nz;
                }
                nbrput()[f] = q;
            }
        }
        consumer_sync(C::NT);
        nl_ = misc()[0];
        fast_ = x0 + TX <= nx && y0 + TY <= ny;
        zloc_lo_ = 1 << 30;
        zloc_hi_ = -1;
        for (int e = 0; e < nl_; ++e) {
            const int zq = loc()[e].z;
            zloc_lo_ = min(zloc_lo_, zq);
            zloc_hi_ = max(zloc_hi_, zq);
        }
        ust = unext + (size_t)(z0 + R) * plane_ + roff_[0];
        wdelta = DELTA ? (long long)(wbuf - unext) : 0;
    }

    __device__ __forceinline__ void end_item(int it)
    {
        double v = (double)nacc + (double)ncomp;
        if (SCALED) v *= (double)isu_ * (double)isu_;   // sums of (su u)^2
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red()[tid >> 5] = v;
        consumer_sync(C::NT);
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < C::NCW; ++w) s += red()[w];
            A.partials[(size_t)kk * A.nitems + it] = s;
        }
    }

    // ---- arithmetic of one row of 4 points ---------------------------
    // P is the plane's phase within a trip of the z loop: its z neighbours
    // sit at queue entries R + P - m and R + P + m.  With PK the arithmetic
    // runs on aligned float2 pairs, each lane rounded once to nearest, which
    // gives the same bits as the scalar order; the x pair sums at even
    // distances are aligned pairs too (x[2h - m], x[2h + 1 - m]) +
    // (x[2h + m], x[2h + 1 + m]), those at odd distances straddle the pairs
    // and stay scalar.
    template <int P>
    __device__ __forceinline__ void laplacian_row(const G (&yv)[PY + 8], const G &lf,
                                                  const G &rt, int r, G &out)
    {
        constexpr int c = R + P;
        M sx[5][4];
#pragma unroll
        for (int m = 1; m <= 4; ++m)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (PK && (m & 1) == 0) continue;    // packed below
                M xm = (i - m >= 0) ? yv[r + R].get(i - m) : lf.get(4 + i - m);
                M xp = (i + m <= 3) ? yv[r + R].get(i + m) : rt.get(i + m - 4);
                sx[m][i] = add_rn(xm, xp);
            }
        if constexpr (PK) {
            // aligned x pairs k = -4, -2, 0, 2, 4, 6 of this row
            auto xpair = [&](int k) -> float2 {
                return k < 0 ? lf.pair((k + 4) >> 1)
                             : (k < 4 ? yv[r + R].pair(k >> 1) : rt.pair((k - 4) >> 1));
            };
            const float2 c0 = make_float2(W<M>::c0x3, W<M>::c0x3);
            const float2 c1 = make_float2(W<M>::c1, W<M>::c1);
            const float2 c2 = make_float2(W<M>::c2, W<M>::c2);
            const float2 c3 = make_float2(W<M>::c3, W<M>::c3);
            const float2 c4 = make_float2(W<M>::c4, W<M>::c4);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 S[5];
#pragma unroll
                for (int m = 1; m <= 4; ++m) {
                    float2 sy = __fadd2_rn(yv[r + R - m].pair(h), yv[r + R + m].pair(h));
                    float2 sz = __fadd2_rn(Q[c - m][r].pair(h), Q[c + m][r].pair(h));
                    const float2 sxp = (m & 1) ? make_float2(sx[m][2 * h], sx[m][2 * h + 1])
                                               : __fadd2_rn(xpair(2 * h - m), xpair(2 * h + m));
                    S[m] = __fadd2_rn(__fadd2_rn(sxp, sy), sz);
                }
                float2 l = __ffma2_rn(c1, S[1], __fmul2_rn(c0, yv[r + R].pair(h)));
                l = __ffma2_rn(c2, S[2], l);
                l = __ffma2_rn(c3, S[3], l);
                l = __ffma2_rn(c4, S[4], l);
                if (h) out.b = l; else out.a = l;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                M s[5];
#pragma unroll
                for (int m = 1; m <= 4; ++m)
                    s[m] = add_rn(add_rn(sx[m][i], add_rn(yv[r + R - m].get(i), yv[r + R + m].get(i))),
                                  add_rn(Q[c - m][r].get(i), Q[c + m][r].get(i)));
                M l = fma_rn(W<M>::c1, s[1], mul_rn(W<M>::c0x3, yv[r + R].get(i)));
                l = fma_rn(W<M>::c2, s[2], l);
                l = fma_rn(W<M>::c3, s[3], l);
                l = fma_rn(W<M>::c4, s[4], l);
                out.set(i, l);
            }
        }
    }

    // 3-level: u' = G (2u - G u_prev + coef lap);
    // delta:   w' = G (w + coef lap),  u' = G u + w'.
    // Delta storage holds U = su u and W = sw w with power-of-two scales, and
    // the arithmetic runs on the stored values: lap(U) = su lap(u), so
    // W' = G (W + (q coef) lap(U)) and U' = G U + W' / q with q = sw / su.
    // Multiplying by a power of two is exact, so this gives the bits of the
    // unscaled formulas scaled; BF16 storage is unscaled (q = 1).
    __device__ __forceinline__ void update_row(const G &u, const G &pa, const G &cf,
                                               const G &lap, const G &gxy, M gz,
                                               G &un, G &wn)
    {
        if constexpr (PK) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 U = u.pair(h), Pp = pa.pair(h), L = lap.pair(h);
                float2 CF = cf.pair(h);
                float2 Gs = make_float2(1.0f, 1.0f);
                if (SPONGE) Gs = __fmul2_rn(gxy.pair(h), make_float2(gz, gz));
                float2 UN, WN = make_float2(0.0f, 0.0f);
                if (DELTA) {
                    if (SCALED) CF = __fmul2_rn(CF, make_float2(q_, q_));
                    const float2 a = __ffma2_rn(CF, L, Pp);
                    WN = SPONGE ? __fmul2_rn(Gs, a) : a;
                    const float2 wq = SCALED ? __fmul2_rn(WN, make_float2(iq_, iq_)) : WN;
                    UN = SPONGE ? __ffma2_rn(Gs, U, wq) : __fadd2_rn(U, wq);
                } else {
                    // 2u - G u_prev rounded once: fma(-G, u_prev, u + u)
                    const float2 nG = SPONGE ? make_float2(-Gs.x, -Gs.y)
                                             : make_float2(-1.0f, -1.0f);
                    const float2 tt = __ffma2_rn(nG, Pp, __fadd2_rn(U, U));
                    const float2 a = __ffma2_rn(CF, L, tt);
                    UN = SPONGE ? __fmul2_rn(Gs, a) : a;
                }
                if (h) { un.b = UN; wn.b = WN; } else { un.a = UN; wn.a = WN; }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                M Gs = SPONGE ? mul_rn(gxy.get(i), gz) : M(1);
                if (DELTA) {
                    M c = SCALED ? mul_rn(cf.get(i), q_) : cf.get(i);
                    M a = fma_rn(c, lap.get(i), pa.get(i));
                    M wv = SPONGE ? mul_rn(Gs, a) : a;
                    M wq = SCALED ? mul_rn(wv, iq_) : wv;
                    wn.set(i, wv);
                    un.set(i, SPONGE ? fma_rn(Gs, u.get(i), wq) : add_rn(u.get(i), wq));
                } else {
                    M tt = fma_rn(-Gs, pa.get(i), add_rn(u.get(i), u.get(i)));
                    M a = fma_rn(cf.get(i), lap.get(i), tt);
                    un.set(i, SPONGE ? mul_rn(Gs, a) : a);
                    wn.set(i, M(0));
                }
            }
        }
    }

    // sum of u'^2 over this thread's valid points of one row into the
    // plane's partials (pp: packed lanes, ps: scalar)
    __device__ __forceinline__ void accumulate_norm(const G &un, float2 &pp, M &ps)
    {
        if constexpr (PK) {
            if (vx == 4) {
                pp = __ffma2_rn(un.a, un.a, pp);
                pp = __ffma2_rn(un.b, un.b, pp);
                return;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < vx) ps = fma_rn(un.get(i), un.get(i), ps);
    }

    // the plane's partial sum of squares x into the pair (nacc, ncomp):
    // TwoSum gives nacc + x = t + e exactly, e is added to the compensation
    __device__ __forceinline__ void add_plane_norm(const float2 &pp, M ps)
    {
        M x = ps;
        if constexpr (PK) x = add_rn(add_rn(pp.x, pp.y), ps);
        const M t = add_rn(nacc, x);
        const M bp = add_rn(t, -nacc);
        const M e = add_rn(add_rn(nacc, -add_rn(t, -bp)), add_rn(x, -bp));
        nacc = t;
        ncomp = add_rn(ncomp, e);
    }

    // ---- the z loop of one item --------------------------------------
    // Queue entries 0..7 hold this thread's points on the 8 planes before the
    // one that arrives; the arriving plane lands in entry 8 + P (P = phase
    // within a trip of KP planes) and the compute plane is the one 4 back.

    // one more u plane consumed: tg and its ring position
    __device__ __forceinline__ void advance_u()
    {
        ++tg;
        if (++us == SU) {
            us = 0;
            uph ^= 1u;
        }
    }

    // Fill: the item's first 8 planes (interior z0 - 4 .. z0 + 3) only enter
    // the queue.  Each plane load is handed back 4 loads later.
    template <int QI>
    __device__ __forceinline__ void fill_one()
    {
        wait_or_abort(ufull(us), uph);
        const T *pl = ubuf(us);
#pragma unroll
        for (int r = 0; r < PY; ++r)
            ld_grp<T, PK>(pl + (PY * ty + r + R) * C::RW + HL + 4 * tx, Q[QI][r]);
        __syncwarp();
        if (tg >= R) {
            if (lane == 0) mbar_arrive(uempty(cs));
            cs = cs + 1 == SU ? 0 : cs + 1;
        }
        advance_u();
    }

    // One compute plane z.  FAST: a whole tile (every row and point valid)
    // with no halo puts, sources or receivers.
    template <int P, bool FAST, bool LOC>
    __device__ __forceinline__ void step_plane(int z)
    {
        // (1) x/y neighbours from the compute plane, staged R loads ago (its
        // full barrier was waited on then): issued before the waits below
        const T *pl = ubuf(cs);
        G yv[PY + 8], lf[PY], rt[PY];
        // the thread's own rows of the compute plane are already in the
        // queue (entry R + P, the same bits); only the y neighbours load
#pragma unroll
        for (int j = 0; j < PY + 8; ++j) {
            if (j >= R && j < R + PY) yv[j] = Q[R + P][j - R];
            else ld_grp<T, PK>(pl + (PY * ty + j) * C::RW + HL + 4 * tx, yv[j]);
        }
#pragma unroll
        for (int r = 0; r < PY; ++r) {
            const T *row = pl + (PY * ty + r + R) * C::RW + HL + 4 * tx;
            ld_grp<T, PK>(row - 4, lf[r]);
            ld_grp<T, PK>(row + 4, rt[r]);
        }
        // (2) the plane that arrives now: the z + 4 neighbours
        {
            wait_or_abort(ufull(us), uph);
            const T *pn = ubuf(us);
#pragma unroll
            for (int r = 0; r < PY; ++r)
                ld_grp<T, PK>(pn + (PY * ty + r + R) * C::RW + HL + 4 * tx, Q[8 + P][r]);
        }
        // (3) the pointwise tiles of plane z
        const unsigned ps = pss;
        wait_or_abort(pfull(ps), pph);
        G pa[PY], cf[PY];
#pragma unroll
        for (int r = 0; r < PY; ++r) {
            ld_grp<T, PK>(pbuf(ps, 0) + (PY * ty + r) * TX + 4 * tx, pa[r]);
            ld_grp<typename C::CT, PK>(
                reinterpret_cast<const typename C::CT *>(pbuf(ps, 1)) +
                    (PY * ty + r) * TX + 4 * tx, cf[r]);
        }
        M gz = M(1);
        if (SPONGE) {
            gz = gz_next;                       // loaded one plane ago
            if (z + 1 < z1) gz_next = (M)__ldg(gz_ptr + z + 1);
        }
        G lap[PY];
#pragma unroll
        for (int r = 0; r < PY; ++r) laplacian_row<P>(yv, lf[r], rt[r], r, lap[r]);
        // sources and receivers: only on the planes that hold some (fast
        // items with puts have none)
        const bool locz = LOC && z >= zloc_lo_ && z <= zloc_hi_;
        if (locz) add_sources(z, lap);
        // leapfrog update with the sponge
        G un[PY], wn[PY];
#pragma unroll
        for (int r = 0; r < PY; ++r)
            update_row(yv[r + R], pa[r], cf[r], lap[r], gxy[r], gz, un[r], wn[r]);
        // stores: u' (and w') at this plane; norm partial
        float2 nrm2 = make_float2(0.0f, 0.0f);   // this plane's sum of u'^2
        M nrm = M(0);
#pragma unroll
        for (int r = 0; r < PY; ++r) {
            T *up = ust + r * (long long)px_;
            M so[4], sw[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                so[i] = un[r].get(i);
                sw[i] = wn[r].get(i);
            }
            if (FAST) {
                if constexpr (PK) {
                    nrm2 = __ffma2_rn(un[r].a, un[r].a, nrm2);
                    nrm2 = __ffma2_rn(un[r].b, un[r].b, nrm2);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) nrm = fma_rn(so[i], so[i], nrm);
                }
                S::st4(up, so);
                if (DELTA) S::st4(up + wdelta, sw);
                continue;
            }
            if (!rowok[r] || vx == 0) continue;
            accumulate_norm(un[r], nrm2, nrm);
            if (vx == 4) {
                S::st4(up, so);
                if (DELTA) S::st4(up + wdelta, sw);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i < vx) {
                        S::st1(up + i, so[i]);
                        if (DELTA) S::st1(up + wdelta + i, sw[i]);
                    }
                }
            }
        }
        add_plane_norm(nrm2, nrm);
        if (locz) record_receivers(z, un);
        ust += plane_;
        // (4) hand slots back: the compute plane's load (its last use) and
        // the pointwise tiles
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(uempty(cs));
            mbar_arrive(pempty(ps));
        }
        cs = cs + 1 == SU ? 0 : cs + 1;
        if (++pss == SP) {
            pss = 0;
            pph ^= 1u;
        }
        ++jg;
        advance_u();
    }

    // point sources: lap += wavelet[n] at the source cell, in the stored
    // scale (the loop only finds the point; the add is a select over
    // compile-time indices, so lap stays in registers)
    __device__ __forceinline__ void add_sources(int z, G (&lap)[PY])
    {
        const int nl = nl_;
        for (int e = 0; e < nl; ++e) {
            int4 q = loc()[e];
            if (q.x < 0 && q.z == z) {
                int lx = q.y & 0xffff, ly = q.y >> 16;
                if ((lx >> 2) == tx && ly / PY == ty && n < cap_) {
                    const int k = (ly % PY) * 4 + (lx & 3);
                    M wv = (M)__ldg(sh->wavelet + (size_t)(-1 - q.x) * cap_ + n);
                    if (SCALED) wv = mul_rn(wv, (M)sh->su);
#pragma unroll
                    for (int r = 0; r < PY; ++r)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            lap[r].set(i, (k == r * 4 + i) ? add_rn(lap[r].get(i), wv) : lap[r].get(i));
                }
            }
        }
    }

    // receivers: trace[n] = u_{n+1} (unscaled)
    __device__ __forceinline__ void record_receivers(int z, const G (&un)[PY])
    {
        const int nl = nl_;
        for (int e = 0; e < nl; ++e) {
            int4 q = loc()[e];
            if (q.x >= 0 && q.z == z) {
                int lx = q.y & 0xffff, ly = q.y >> 16;
                if ((lx >> 2) == tx && ly / PY == ty && n < cap_) {
                    const int k = (ly % PY) * 4 + (lx & 3);
                    M v = M(0);
#pragma unroll
                    for (int r = 0; r < PY; ++r)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            v = (k == r * 4 + i) ? un[r].get(i) : v;
                    if (SCALED) v = mul_rn(v, isu_);
                    sh->traces[(size_t)q.x * cap_ + n] = (float)v;
                }
            }
        }
    }

    __device__ __forceinline__ void shift_queue()
    {
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int r = 0; r < PY; ++r) Q[q][r] = Q[q + KP][r];
    }

    // the compute planes of one item, KP per trip of the loop
    template <bool FAST, bool LOC>
    __device__ __forceinline__ void z_loop(int nzc)
    {
#pragma unroll 1
        for (int tb = 0; tb < nzc; tb += KP) {
            step_plane<0, FAST, LOC>(z0 + tb);
            if (tb + 1 < nzc) step_plane<1, FAST, LOC>(z0 + tb + 1);
            if constexpr (KP > 2) {
                if (tb + 2 < nzc) step_plane<2, FAST, LOC>(z0 + tb + 2);
                if (tb + 3 < nzc) step_plane<3, FAST, LOC>(z0 + tb + 3);
            }
            shift_queue();
        }
    }

    // ---- fused halo puts (Listing 1's ompx_put, done by the step kernel) --
    // After the item's z loop and a consumer barrier (which orders every
    // consumer thread's stores of the item before the loads below), the
    // consumer threads copy the item's boundary strips of u_{n+1} -- at most
    // R cells deep along each face that has a neighbour -- from this
    // subdomain's field, where they were just stored and still sit in L2,
    // into the face neighbours' halos.  The z loop of a boundary item is
    // then the same as an interior item's (per-row put code in the loop
    // cost 16-45 % in instruction issue and fetch).

    // 4 elements of T moved as one unit: 16 bytes (FP32), 8 (16-bit) or
    // 2 x 16 (FP64), through L2 only (the source was stored moments ago by
    // other threads of this CTA; nothing of it is in L1)
    struct Vec4 {
        using W = typename std::conditional<sizeof(T) == 2, uint2, uint4>::type;
        W a, b;
        __device__ __forceinline__ void load(const T *p)
        {
            a = __ldcg(reinterpret_cast<const W *>(p));
            if constexpr (sizeof(T) == 8) b = __ldcg(reinterpret_cast<const W *>(p) + 1);
        }
        __device__ __forceinline__ void store(T *p) const
        {
            __stcg(reinterpret_cast<W *>(p), a);
            if constexpr (sizeof(T) == 8) __stcg(reinterpret_cast<W *>(p) + 1, b);
        }
    };

    // What the puts of one item need (passed by value, so that the put code
    // can live out of line without putting the Step object in memory).
    struct PutItem {
        T *u;                  // this subdomain's u_{n+1}
        const NbrPut *nbr;     // per face: the neighbour's buffer and strides
        size_t plane;          // this subdomain's plane stride
        int px;                // and row pitch
        int x0, y0, z0, z1, nx, ny, nz;
        int has;               // bit f: face f has a neighbour
    };

    __device__ __noinline__ static void put_item(const PutItem p, int tid)
    {
        constexpr int B = sizeof(T) == 8 ? 4 : 8;   // copies in flight per thread
        const int xe = min(p.x0 + TX, p.nx), ye = min(p.y0 + TY, p.ny);
        for (int f = 0; f < 6; ++f) {
            if (!(p.has >> f & 1)) continue;
            // the part of this item within R of face f, and where it goes
            int xl = p.x0, xh = xe, yl = p.y0, yh = ye, zl = p.z0, zh = p.z1;
            int dx = 0, dy = 0, dz = 0;
            const NbrPut q = p.nbr[f];
            switch (f) {
            case 0: xh = min(xh, R); dx = q.ext; break;        // -> its +x halo
            case 1: xl = max(xl, p.nx - R); dx = -p.nx; break; // -> its -x halo
            case 2: yh = min(yh, R); dy = q.ext; break;
            case 3: yl = max(yl, p.ny - R); dy = -p.ny; break;
            case 4: zh = min(zh, R); dz = q.ext; break;
            default: zl = max(zl, p.nz - R); dz = -p.nz; break;
            }
            if (xl >= xh || yl >= yh || zl >= zh) continue;
            const T *src0 = p.u + (size_t)(zl + R) * p.plane + (size_t)(yl + R) * p.px + XO + xl;
            T *dst0 = reinterpret_cast<T *>(q.base) + (long long)(zl + dz + R) * q.plane +
                      (long long)(yl + dy + R) * q.px + XO + xl + dx;
            const int rows = yh - yl, xw = xh - xl;
            // rows of the box in chunks of 4 elements (the last may be short)
            const int nch = (xw + 3) / 4;
            const int units = (zh - zl) * rows * nch;
            // whole chunks starting on 4-element boundaries on both sides:
            // vector units (all of them, except at x cuts off that grid)
            const bool vec = (xw & 3) == 0 && ((XO + xl) & 3) == 0 &&
                             ((XO + xl + dx) & 3) == 0;
            for (int u0 = tid; u0 < units; u0 += B * C::NT) {
                Vec4 v[B];
                T *d[B];
                const T *sp[B];
                int n[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const int u = u0 + k * C::NT;
                    d[k] = nullptr;
                    sp[k] = nullptr;
                    n[k] = 0;
                    if (u < units) {
                        const int ch = u % nch, row = u / nch;
                        const int y = row % rows, z = row / rows;
                        sp[k] = src0 + (size_t)z * p.plane + (size_t)y * p.px + 4 * ch;
                        d[k] = dst0 + (long long)z * q.plane + (long long)y * q.px + 4 * ch;
                        n[k] = min(4, xw - 4 * ch);
                        if (vec) v[k].load(sp[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    if (!d[k]) continue;
                    if (vec) v[k].store(d[k]);
                    else
                        for (int i = 0; i < n[k]; ++i) d[k][i] = sp[k][i];
                }
            }
        }
    }

    __device__ __forceinline__ void run()
    {
        tid = threadIdx.x;
        lane = tid & 31;
        if (tid == 0) {
            for (int q = 0; q < SU; ++q) {
                mbar_init(ufull(q), 1);
                mbar_init(uempty(q), C::NCW);
            }
            for (int q = 0; q < SP; ++q) {
                mbar_init(pfull(q), 1);
                mbar_init(pempty(q), C::NCW);
            }
            for (int q = 0; q < C::IQ; ++q) {
                mbar_init(iqfull(q), 1);
                mbar_init(iqempty(q), 1);
            }
            misc()[1] = 0;
            fence_barrier_init();
        }
        __syncthreads();
        if (tid >= C::NT) {            // the producer warp
            if (tid == C::NT) produce();
            return;
        }
        tx = tid % C::NTX;
        ty = tid / C::NTX;
        aborted = false;
        tg = jg = 0;
        us = uph = cs = pss = pph = 0;
        itn_ = 0;
        for (int k = 0; k < A.nk; ++k) {
            kk = A.k + k;
            for (;;) {
                const int it = next_item();
                if (it == -2) return;      // this CTA gave up (error bit set)
                if (it < 0) break;
                begin_item(it);
                fill_one<0>(); fill_one<1>(); fill_one<2>(); fill_one<3>();
                fill_one<4>(); fill_one<5>(); fill_one<6>(); fill_one<7>();
                // three loop bodies, so that each item runs the smallest
                // code that covers it (instruction fetch limits the loop):
                // whole tiles without sources/receivers, whole tiles with
                // sources/receivers on some planes, and partial tiles.  The
                // source/receiver code in the main body cost 7-9 % with
                // 16-bit storage; partial tiles on a body with per-row
                // checks and per-point masks everywhere cost 16 % at 1200^3.
                // Halo puts run after the loop (put_item).
                if (fast_ && nl_ == 0) z_loop<true, false>(z1 - z0);
                else if (fast_) z_loop<true, true>(z1 - z0);
                else z_loop<false, true>(z1 - z0);
                if (item_puts) {           // uniform over the CTA
                    consumer_sync(C::NT);
                    PutItem p;
                    p.u = unext;
                    p.nbr = nbrput();
                    p.plane = plane_;
                    p.px = px_;
                    p.x0 = x0; p.y0 = y0; p.z0 = z0; p.z1 = z1;
                    p.nx = nx; p.ny = ny; p.nz = nz;
                    p.has = 0;
#pragma unroll
                    for (int f = 0; f < 6; ++f) p.has |= (nbr_[f] >= 0 ? 1 : 0) << f;
                    put_item(p, tid);
                }
                end_item(it);
            }
            if (k + 1 < A.nk) {
                // arrive at the device-wide barrier once this CTA's stores of
                // the step (interior and halo puts) are visible
                __threadfence();
                fence_proxy_async_global();
                consumer_sync(C::NT);
                if (tid == 0) red_release_gpu_add(A.gbar, 1u);
            }
        }
    }
};

template <class C, bool DELTA, bool SPONGE>
__global__ void __maxnreg__(C::MAXREG)
k_step(const __grid_constant__ StepArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    Step<C, DELTA, SPONGE> s(a, smem);
    s.run();
}

template <class C>
static TileInfo info_of()
{
    return TileInfo{C::TX, C::TY, C::THREADS, (size_t)C::SMEM};
}

template <class C, bool DELTA>
static cudaError_t launch_cfg(bool sponge, int grid, const StepArgs &a,
                              cudaStream_t s)
{
    auto kern = sponge ? k_step<C, DELTA, true> : k_step<C, DELTA, false>;
    static bool attr_done[2] = {false, false};
    if (!attr_done[sponge]) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr_done[sponge] = true;
    }
    if (a.nk <= 1) {
        kern<<<grid, C::THREADS, C::SMEM, s>>>(a);
        return cudaGetLastError();
    }
    // several steps in one launch: the CTAs wait for each other between
    // steps, so they must all be resident (cooperative launch)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class C, bool DELTA>
static int occ_cfg(bool sponge)
{
    auto kern = sponge ? k_step<C, DELTA, true> : k_step<C, DELTA, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             C::SMEM) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::THREADS,
                                                      C::SMEM) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace gw
