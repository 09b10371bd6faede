// aux_kernels.cu -- the kernels around the fused step: model precompute
// (vmax, coef = (v dt / h)^2 in FP64), dense <-> padded field transfers,
// the separate face-halo put (pack/put/unpack of Listing 1, section 4.5),
// the end-of-chunk FP64 norm reduction, and the FP64 energy check.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "check_sums.cuh"
#include "gw_device.h"
#include "gw_kernels.h"

namespace gw {

// ---------------------------------------------------------------- scalars

template <class T> __device__ __forceinline__ double to_d(T v);
template <> __device__ __forceinline__ double to_d<float>(float v) { return v; }
template <> __device__ __forceinline__ double to_d<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_d<__half>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

__device__ __forceinline__ size_t pidx(const SubDev &s, int xo, int x, int y, int z)
{
    return ((size_t)(z + R) * s.py + (size_t)(y + R)) * s.px + (size_t)(xo + x);
}

// ---------------------------------------------------------------- vmax

// Max over a dense slab, compared in the input's own type (the max of FP32
// values is one of them, so comparing FP32 values in FP32 gives the same
// result as comparing them in FP64, at FP32 speed).
template <class V>
__global__ void k_vmax(const V *v, size_t n, unsigned long long *out)
{
    V m = V(0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const V x = v[i];
        m = x > m ? x : m;     // a NaN never wins
    }
    double md = (double)m;
    for (int o = 16; o > 0; o >>= 1) {
        double t = __shfl_xor_sync(0xffffffffu, md, o);
        md = t > md ? t : md;
    }
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && md > 0.0)
        atomicMax(out, (unsigned long long)__double_as_longlong(md));
}

cudaError_t launch_vmax(const void *v, size_t n, int f32,
                        unsigned long long *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    grid = grid > 4096 ? 4096 : grid;
    if (f32)
        k_vmax<float><<<grid, 256, 0, s>>>(static_cast<const float *>(v), n, out);
    else
        k_vmax<double><<<grid, 256, 0, s>>>(static_cast<const double *>(v), n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- coef

// Exact FP32 -> FP64 and round-to-nearest-even FP64 -> FP32 conversions in
// integer arithmetic, for normal numbers (IEEE 754 binary32 / binary64:
// rebias the exponent, move the significand; for the narrowing, round the
// 29 dropped significand bits half to even, carrying into the exponent).
// Anything else -- zero, subnormal, infinite, NaN, out of FP32's normal
// range -- takes the hardware conversion.  GB300's FP64 pipe is narrow and
// conversions to and from FP64 run on it, so the coefficient square below
// spends it on its two products only.
__device__ __forceinline__ double f32_to_f64(float v)
{
    const uint32_t u = __float_as_uint(v);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)v;
    const uint64_t b = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e - 127u + 1023u) << 52) |
                       ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int fe = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
    if (fe <= 0 || fe >= 0xff) return (float)x;
    const uint64_t m = b & ((1ull << 52) - 1ull);
    uint32_t r = (uint32_t)(m >> 29);
    const uint64_t rest = m & ((1ull << 29) - 1ull), half = 1ull << 28;
    uint32_t ex = (uint32_t)fe;
    if (rest > half || (rest == half && (r & 1u))) {
        if (++r == (1u << 23)) {
            r = 0u;
            if (++ex == 0xffu) return (float)x;     // rounds to infinity
        }
    }
    return __uint_as_float((uint32_t)(b >> 63) << 31 | ex << 23 | r);
}

// coef of one input value: (v dt/h)^2 formed in FP64 and rounded to the
// coef type, or (raw) v itself
template <class CT, class V> struct CoefOf {
    __device__ __forceinline__ static CT get(V v, double dt_over_h, int raw)
    {
        const double nu = (double)v * dt_over_h;   // FP64 precompute
        return from_d<CT>(raw ? (double)v : nu * nu);
    }
};
template <> struct CoefOf<float, float> {
    __device__ __forceinline__ static float get(float v, double dt_over_h, int raw)
    {
        if (raw) return v;
        const double nu = f32_to_f64(v) * dt_over_h;
        return f64_to_f32_rn(nu * nu);
    }
};

// the narrowing conversion above over a device array (the library's
// conversion pinned against IEEE round-to-nearest-even by the tests)
__global__ void k_round_to_f32(const double *in, float *out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = f64_to_f32_rn(in[i]);
}

cudaError_t launch_round_to_f32(const double *in, float *out, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int g = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_round_to_f32<<<g, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// One block per row (y, z) of the slab's planes inside the subdomain at a
// time, threads along x: no per-element index division.
template <class CT, class V>
__global__ void k_coef(ModelSlab m, SubDev sd, int xo)
{
    // planes of the slab inside this subdomain
    const int zl = max(m.z_lo, sd.gz0), zh = min(m.z_hi, sd.gz0 + sd.nz);
    if (zl >= zh) return;
    const unsigned ny = (unsigned)sd.ny, rows = ny * (unsigned)(zh - zl);
    const V *v = static_cast<const V *>(m.v);
    CT *c = reinterpret_cast<CT *>(sd.coef);
    for (unsigned r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % ny), gz = zl + (int)(r / ny);
        CT *row = c + pidx(sd, xo, 0, y, gz - sd.gz0);
        if (m.layered) {
            const CT cv = CoefOf<CT, V>::get(v[gz - m.z_lo], m.dt_over_h, m.raw);
            for (int x = threadIdx.x; x < sd.nx; x += blockDim.x) row[x] = cv;
        } else {
            const V *src = v + ((size_t)(gz - m.z_lo) * m.NY + (size_t)(sd.gy0 + y)) * m.NX +
                           (size_t)sd.gx0;
            for (int x = threadIdx.x; x < sd.nx; x += blockDim.x)
                row[x] = CoefOf<CT, V>::get(src[x], m.dt_over_h, m.raw);
        }
    }
}

// coef = (v dt / h)^2 over a subdomain whose coef array holds v (exactly:
// only used when the coef type holds the input velocities without
// rounding): the same FP64 products, so the same bits as k_coef from the
// input
template <class CT>
__global__ void k_coef_square(SubDev sd, int xo, double dt_over_h)
{
    CT *c = reinterpret_cast<CT *>(sd.coef);
    const unsigned ny = (unsigned)sd.ny, rows = ny * (unsigned)sd.nz;
    for (unsigned r = blockIdx.x; r < rows; r += gridDim.x) {
        CT *row = c + pidx(sd, xo, 0, (int)(r % ny), (int)(r / ny));
        for (int x = threadIdx.x; x < sd.nx; x += blockDim.x)
            row[x] = CoefOf<CT, CT>::get(row[x], dt_over_h, 0);
    }
}

static int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    return (int)(g > 8192 ? 8192 : (g ? g : 1));
}

// blocks for a row walk: one row per block at a time, at most 8 blocks per
// SM's worth (152 SMs)
static int grid_rows(size_t rows)
{
    return (int)std::min<size_t>(std::max<size_t>(rows, 1), 152 * 8);
}

cudaError_t launch_coef_square(const SubDev &sd, int dtype, double dt_over_h,
                               cudaStream_t s)
{
    if ((size_t)sd.ny * sd.nz > 0xffffffffull) return cudaErrorInvalidValue;
    const int g = grid_rows((size_t)sd.ny * sd.nz);
    const int xo = dtype_xoff(dtype);
    switch (dtype) {
    case DT_F32: k_coef_square<float><<<g, 256, 0, s>>>(sd, xo, dt_over_h); break;
    case DT_F64: k_coef_square<double><<<g, 256, 0, s>>>(sd, xo, dt_over_h); break;
    default: return cudaErrorInvalidValue;   // FP16 coef cannot hold v exactly
    }
    return cudaGetLastError();
}

cudaError_t launch_coef(const ModelSlab &m, const SubDev &sd, int dtype,
                        cudaStream_t s)
{
    if ((size_t)sd.ny * (size_t)(m.z_hi - m.z_lo) > 0xffffffffull) return cudaErrorInvalidValue;
    const int g = grid_rows((size_t)sd.ny * (size_t)(m.z_hi - m.z_lo));
    const int xo = dtype_xoff(dtype);
#define GW_COEF(CT)                                                     \
    (m.f32 ? (k_coef<CT, float><<<g, 256, 0, s>>>(m, sd, xo), 0)        \
           : (k_coef<CT, double><<<g, 256, 0, s>>>(m, sd, xo), 0))
    switch (dtype) {
    case DT_F32: GW_COEF(float); break;
    case DT_F64: GW_COEF(double); break;
    default: GW_COEF(__half); break;   // reduced storage keeps coef in FP16
    }
#undef GW_COEF
    return cudaGetLastError();
}

// ---------------------------------------------------------------- transfers

template <class T, class D, bool SCATTER>
__global__ void k_xfer(FieldSlab f, SubDev sd, int xo)
{
    int zl = max(f.z_lo, sd.gz0), zh = min(f.z_hi, sd.gz0 + sd.nz);
    if (zl >= zh) return;
    size_t npl = (size_t)sd.nx * sd.ny;
    size_t n = npl * (size_t)(zh - zl);
    char *base = f.which == 0 ? sd.u[f.cur] : f.which == 1 ? sd.u[f.cur ^ 1]
               : f.which == 2 ? sd.w : sd.coef;
    T *a = reinterpret_cast<T *>(base);
    D *d = static_cast<D *>(f.dense);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % sd.nx);
        int y = (int)((i / sd.nx) % sd.ny);
        int gz = zl + (int)(i / npl);
        size_t di = ((size_t)(gz - f.z_lo) * f.NY + (size_t)(sd.gy0 + y)) * f.NX +
                    (size_t)(sd.gx0 + x);
        size_t pi = pidx(sd, xo, x, y, gz - sd.gz0);
        if (SCATTER)
            a[pi] = from_d<T>((double)d[di] * f.scale);
        else
            d[di] = (D)(to_d<T>(a[pi]) / f.scale);
    }
}

template <bool SCATTER>
static cudaError_t xfer(const FieldSlab &f, const SubDev &sd, int dtype,
                        cudaStream_t s)
{
    size_t n = (size_t)sd.nx * sd.ny * (size_t)(f.z_hi - f.z_lo);
    int g = grid_for(n);
    int xo = dtype_xoff(dtype);
    bool coef = f.which == 3;
#define GW_X(T)                                                              \
    (f.f64 ? (k_xfer<T, double, SCATTER><<<g, 256, 0, s>>>(f, sd, xo), 0)    \
           : (k_xfer<T, float, SCATTER><<<g, 256, 0, s>>>(f, sd, xo), 0))
    switch (dtype) {
    case DT_F32: GW_X(float); break;
    case DT_F64: GW_X(double); break;
    case DT_F16S: if (coef) GW_X(__half); else GW_X(__half); break;
    case DT_BF16: if (coef) GW_X(__half); else GW_X(__nv_bfloat16); break;
    default: return cudaErrorInvalidValue;
    }
#undef GW_X
    return cudaGetLastError();
}

cudaError_t launch_scatter(const FieldSlab &f, const SubDev &sd, int dtype,
                           cudaStream_t s)
{
    return xfer<true>(f, sd, dtype, s);
}

cudaError_t launch_gather(const FieldSlab &f, const SubDev &sd, int dtype,
                          cudaStream_t s)
{
    return xfer<false>(f, sd, dtype, s);
}

// ---------------------------------------------------------------- halo put

// Element counts and the source/destination boxes of one face copy.
__device__ __forceinline__ void face_box(const SubDev &s, const SubDev &d,
                                         int face, int &ex, int &ey, int &ez,
                                         int &sx, int &sy, int &sz, int &dx,
                                         int &dy, int &dz)
{
    ex = s.nx; ey = s.ny; ez = s.nz;
    sx = sy = sz = 0;
    dx = dy = dz = 0;
    switch (face) {
    case 0: ex = R; sx = 0;        dx = d.nx; break;   // -x slab -> nbr's +x halo
    case 1: ex = R; sx = s.nx - R; dx = -R;   break;   // +x slab -> nbr's -x halo
    case 2: ey = R; sy = 0;        dy = d.ny; break;
    case 3: ey = R; sy = s.ny - R; dy = -R;   break;
    case 4: ez = R; sz = 0;        dz = d.nz; break;
    default: ez = R; sz = s.nz - R; dz = -R;  break;
    }
}

// One grid row (blockIdx.y) per face copy; its threads stride over the
// 16-byte units (V elements along x) of that face's box.  A unit whose source
// and destination are both 16-byte aligned moves as one vector; a short or
// misaligned one element by element.
template <class E>
__global__ void k_halo(const HaloDesc *descs, const SubDev *subs, const int *step,
                       int k, int xo)
{
    constexpr int V = 16 / (int)sizeof(E);
    const HaloDesc hd = descs[blockIdx.y];
    const SubDev &s = subs[hd.src];
    const SubDev &d = subs[hd.dst];
    int ex, ey, ez, sx, sy, sz, dx, dy, dz;
    face_box(s, d, hd.face, ex, ey, ez, sx, sy, sz, dx, dy, dz);
    const int buf = (*step + k + 1) & 1;
    const E *src = reinterpret_cast<const E *>(s.u[buf]);
    E *dst = reinterpret_cast<E *>(d.u[buf]);
    const unsigned ux = (unsigned)(ex + V - 1) / V;
    const unsigned units = ux * (unsigned)ey * (unsigned)ez;
    const int fx = hd.face >> 1;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < units;
         i += gridDim.x * blockDim.x) {
        const unsigned row = i / ux;
        const int a = (int)(i - row * ux) * V;
        const int b = (int)(row % (unsigned)ey);
        const int c = (int)(row / (unsigned)ey);
        // the halo cell of d keeps d's own x/y/z for the axes not crossed
        const int tx = fx == 0 ? dx + a : a;
        const int ty = fx == 1 ? dy + b : b;
        const int tz = fx == 2 ? dz + c : c;
        const E *ps = src + pidx(s, xo, sx + a, sy + b, sz + c);
        E *pd = dst + pidx(d, xo, tx, ty, tz);
        const int n = min(V, ex - a);
        if (n == V && ((reinterpret_cast<uintptr_t>(ps) | reinterpret_cast<uintptr_t>(pd)) & 15u) == 0) {
            *reinterpret_cast<uint4 *>(pd) = *reinterpret_cast<const uint4 *>(ps);
        } else {
            for (int q = 0; q < n; ++q) pd[q] = ps[q];
        }
    }
}

cudaError_t launch_halo(const HaloDesc *descs, int ndesc, long long max_units,
                        const SubDev *subs_dev, const int *step, int k,
                        int dtype, cudaStream_t s)
{
    if (max_units <= 0 || ndesc <= 0) return cudaSuccess;
    if (ndesc > 65535 || max_units > 0xffffffffLL) return cudaErrorInvalidValue;
    const int gx = (int)std::min<long long>((max_units + 255) / 256, 1024);
    const dim3 grid(gx, ndesc);
    const int xo = dtype_xoff(dtype);
    switch (dtype_size(dtype)) {
    case 2: k_halo<unsigned short><<<grid, 256, 0, s>>>(descs, subs_dev, step, k, xo); break;
    case 4: k_halo<unsigned int><<<grid, 256, 0, s>>>(descs, subs_dev, step, k, xo); break;
    default: k_halo<unsigned long long><<<grid, 256, 0, s>>>(descs, subs_dev, step, k, xo); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- chunk end

__global__ void k_chunk_end(const ShotDev *shots, const double *partials,
                            int nitems, int nk, unsigned *err)
{
    const ShotDev &sh = shots[blockIdx.x];
    __shared__ double red[256];
    const int n0 = *sh.step;
    // steps from the shot's limit on were skipped: no partials, no count
    const int nk_shot = n0 >= sh.limit ? 0 : min(nk, sh.limit - n0);
    for (int k = 0; k < nk_shot; ++k) {
        const double *p = partials + (size_t)k * nitems + sh.first_item;
        double v = 0.0;
        for (int i = threadIdx.x; i < sh.nitems; i += blockDim.x) v += p[i];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double s = red[0];
            if (n0 + k < sh.cap) sh.norms[n0 + k] = s;
            if (!isfinite(s)) atomicOr(err, ERRB_NONFINITE);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *sh.step = n0 + nk_shot;
}

cudaError_t launch_chunk_end(const ShotDev *shots_dev, int nshots,
                             const double *partials, int nitems, int nk,
                             unsigned *err, cudaStream_t s)
{
    if (nshots <= 0) return cudaSuccess;
    k_chunk_end<<<nshots, 256, 0, s>>>(shots_dev, partials, nitems, nk, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- checks

// One block per interior plane z of a subdomain (check_sums.cuh).
template <class T, class CT>
__global__ void __launch_bounds__(kCheckThreads)
k_check(SubDev sd, int cur, int xo, double isu, double *part)
{
    const int z = blockIdx.x;
    check_plane_sums<T, CT>(reinterpret_cast<const T *>(sd.u[cur]),
                            reinterpret_cast<const T *>(sd.u[cur ^ 1]),
                            reinterpret_cast<const CT *>(sd.coef), sd.nx, sd.ny,
                            (long long)pidx(sd, xo, 0, 0, z), sd.px,
                            (long long)sd.px * sd.py, isu, part + 3 * z);
}

__global__ void __launch_bounds__(kCheckThreads)
k_check_sum(const double *part, int nplanes, double *out)
{
    check_sum_planes(part, nplanes, out);
}

cudaError_t launch_check(const SubDev &sd, int cur, int dtype, double scale_u,
                         double *part, cudaStream_t s)
{
    const int g = sd.nz;
    const int xo = dtype_xoff(dtype);
    const double isu = 1.0 / scale_u;
    switch (dtype) {
    case DT_F32: k_check<float, float><<<g, kCheckThreads, 0, s>>>(sd, cur, xo, isu, part); break;
    case DT_F64: k_check<double, double><<<g, kCheckThreads, 0, s>>>(sd, cur, xo, isu, part); break;
    case DT_F16S: k_check<__half, __half><<<g, kCheckThreads, 0, s>>>(sd, cur, xo, isu, part); break;
    case DT_BF16:
        k_check<__nv_bfloat16, __half><<<g, kCheckThreads, 0, s>>>(sd, cur, xo, isu, part);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_check_sum(const double *part, int nplanes, double *out, cudaStream_t s)
{
    k_check_sum<<<1, kCheckThreads, 0, s>>>(part, nplanes, out);
    return cudaGetLastError();
}

}  // namespace gw
