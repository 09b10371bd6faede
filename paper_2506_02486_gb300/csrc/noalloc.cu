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

#include "check_sums.cuh"
#include "gw_internal.h"

namespace gw {

// Largest nz the scratch array can serve (3 FP64 partials per plane: 96 KiB).
constexpr int kNoallocMaxPlanes = 4096;

static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPlanes * 3];

namespace {

// One block per interior plane z of a caller's padded fields: the same
// sums, in the same order, as gw_check (check_sums.cuh).
template <class T, class CT>
__global__ void __launch_bounds__(kCheckThreads)
k_plane_sums(const T *un, const T *up, const CT *cf, int nx, int ny, int px, int xo,
             double isu, double *part)
{
    const int z = blockIdx.x;
    const long long sy = px, sz = (long long)px * (ny + 2 * R);
    check_plane_sums<T, CT>(un, up, cf, nx, ny, (long long)(z + R) * sz + R * sy + xo, sy, sz,
                            isu, part + 3 * z);
}

__global__ void __launch_bounds__(kCheckThreads)
k_sum_planes(const double *part, int nz, double *out)
{
    check_sum_planes(part, nz, out);
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
        k_plane_sums<float, float><<<nz, kCheckThreads, 0, s>>>(
            static_cast<const float *>(u_cur), static_cast<const float *>(u_prev),
            static_cast<const float *>(coef), nx, ny, px, xo, isu, part);
        break;
    case DT_F64:
        k_plane_sums<double, double><<<nz, kCheckThreads, 0, s>>>(
            static_cast<const double *>(u_cur), static_cast<const double *>(u_prev),
            static_cast<const double *>(coef), nx, ny, px, xo, isu, part);
        break;
    case DT_F16S:
        k_plane_sums<__half, __half><<<nz, kCheckThreads, 0, s>>>(
            static_cast<const __half *>(u_cur), static_cast<const __half *>(u_prev),
            static_cast<const __half *>(coef), nx, ny, px, xo, isu, part);
        break;
    default:
        k_plane_sums<__nv_bfloat16, __half><<<nz, kCheckThreads, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(u_cur),
            static_cast<const __nv_bfloat16 *>(u_prev),
            static_cast<const __half *>(coef), nx, ny, px, xo, isu, part);
        break;
    }
    GW_TRY_CUDA(cudaGetLastError());
    k_sum_planes<<<1, kCheckThreads, 0, s>>>(part, nz, out_dev);
    GW_TRY_CUDA(cudaGetLastError());
    return GW_OK;
}
