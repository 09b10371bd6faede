// noalloc.cu -- gw_check_fields_noalloc: the FP64 check reductions of
// gw_check for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while another
// framework holds its memory pool or allocator lock, an embedded runtime
// that owns every byte of device memory, or a latency-critical path where an
// allocation (which may synchronise the device) is not acceptable.  This
// entry point allocates nothing.  The caller passes the
// three fields and a small output buffer; the per-plane partial sums live in
// the file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gw_internal.h"

namespace gw {

// Largest nz the scratch array can serve (3 FP64 partials per plane: 96 KiB).
constexpr int kNoallocMaxPlanes = 4096;

static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPlanes * 3];

namespace {

template <class T> __device__ __forceinline__ double ld_d(const T *p);
template <> __device__ __forceinline__ double ld_d<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ double ld_d<double>(const double *p) { return *p; }
template <> __device__ __forceinline__ double ld_d<__half>(const __half *p) { return (double)__half2float(*p); }
template <> __device__ __forceinline__ double ld_d<__nv_bfloat16>(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }

// One block per interior plane z: writes (sum u^2, sum (u - up)^2 / coef,
// sum u lap(up)) of that plane to part[3 z .. 3 z + 2].
template <class T, class CT>
__global__ void k_plane_sums(const T *un, const T *up, const CT *cf, int nx,
                             int ny, int px, int xo, double isu, double *part)
{
    const int z = blockIdx.x;
    const double c[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                         -1.0 / 560.0};
    const long long py = ny + 2 * R;
    const long long sy = px, sz = (long long)px * py;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int x = i % nx, y = i / nx;
        const long long p = (long long)(z + R) * sz + (long long)(y + R) * sy + xo + x;
        const double u = ld_d(un + p) * isu;
        const double v = ld_d(up + p) * isu;
        double lap = 3.0 * c[0] * v;
        for (int m = 1; m <= 4; ++m)
            lap += c[m] * (ld_d(up + p - m) + ld_d(up + p + m) + ld_d(up + p - m * sy) +
                           ld_d(up + p + m * sy) + ld_d(up + p - m * sz) +
                           ld_d(up + p + m * sz)) * isu;
        const double d = u - v;
        a0 += u * u;
        a1 += d * d / ld_d(cf + p);
        a2 += u * lap;
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[3 * z + k] = red[k][0];
}

// Sums the plane partials in a fixed order into out[0..2].
__global__ void k_sum_planes(const double *part, int nz, double *out)
{
    __shared__ double red[3][256];
    double a[3] = {0, 0, 0};
    for (int z = threadIdx.x; z < nz; z += blockDim.x)
        for (int k = 0; k < 3; ++k) a[k] += part[3 * z + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k] = red[k][0];
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's host-side name is not a device address).
std::mutex g_addr_mu;
double *g_addr[64] = {nullptr};

gw_status scratch_address(double **out)
{
    int dev = 0;
    GW_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GW_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return GW_OK;
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" gw_status gw_check_fields_noalloc(const void *u_cur, const void *u_prev,
                                             const void *coef, int dtype, int nx,
                                             int ny, int nz, int px, double scale_u,
                                             double *out_dev, gw_stream stream)
{
    if (!u_cur || !u_prev || !coef || !out_dev)
        return fail(GW_ERR_ARG, "NULL field or output pointer");
    if (dtype < DT_F32 || dtype > DT_BF16) return fail(GW_ERR_ARG, "bad dtype %d", dtype);
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(GW_ERR_ARG, "bad grid %d x %d x %d", nx, ny, nz);
    if (nz > kNoallocMaxPlanes)
        return fail(GW_ERR_ARG,
                    "nz = %d exceeds the %d planes the built-in scratch array holds",
                    nz, kNoallocMaxPlanes);
    const int xo = dtype_xoff(dtype);
    if (px < xo + nx + R) return fail(GW_ERR_ARG, "row pitch %d < %d", px, xo + nx + R);
    if (!(scale_u > 0)) return fail(GW_ERR_ARG, "scale_u must be positive");
    double *part = nullptr;
    GW_TRY(scratch_address(&part));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double isu = 1.0 / scale_u;
    switch (dtype) {
    case DT_F32:
        k_plane_sums<float, float><<<nz, 256, 0, s>>>(
            static_cast<const float *>(u_cur), static_cast<const float *>(u_prev),
            static_cast<const float *>(coef), nx, ny, px, xo, isu, part);
        break;
    case DT_F64:
        k_plane_sums<double, double><<<nz, 256, 0, s>>>(
            static_cast<const double *>(u_cur), static_cast<const double *>(u_prev),
            static_cast<const double *>(coef), nx, ny, px, xo, isu, part);
        break;
    case DT_F16S:
        k_plane_sums<__half, __half><<<nz, 256, 0, s>>>(
            static_cast<const __half *>(u_cur), static_cast<const __half *>(u_prev),
            static_cast<const __half *>(coef), nx, ny, px, xo, isu, part);
        break;
    default:
        k_plane_sums<__nv_bfloat16, __half><<<nz, 256, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(u_cur),
            static_cast<const __nv_bfloat16 *>(u_prev),
            static_cast<const __half *>(coef), nx, ny, px, xo, isu, part);
        break;
    }
    GW_TRY_CUDA(cudaGetLastError());
    k_sum_planes<<<1, 256, 0, s>>>(part, nz, out_dev);
    GW_TRY_CUDA(cudaGetLastError());
    return GW_OK;
}
