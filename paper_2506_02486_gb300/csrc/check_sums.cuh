// check_sums.cuh -- the FP64 check reductions shared by gw_check (k_check in
// aux_kernels.cu) and its allocation-free variant (noalloc.cu), so that the
// two compute the same sums in the same order by construction.
//
// One block of kCheckThreads threads per interior plane z: (sum u^2,
// sum (u - up)^2 / coef, sum u lap(up)) of the plane, u and up unscaled by
// isu = 1 / scale_u, in a fixed order (a strided pass over the plane, then a
// shared-memory tree), no atomics, so a check is reproducible bit for bit.
// The discrete energy E = sum (u - up)^2 / coef - sum u lap(up) is the
// conserved quantity of the leapfrog scheme without source and sponge.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gw_device.h"

namespace gw {

constexpr int kCheckThreads = 256;

template <class T> __device__ __forceinline__ double chk_d(const T *p);
template <> __device__ __forceinline__ double chk_d<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ double chk_d<double>(const double *p) { return *p; }
template <> __device__ __forceinline__ double chk_d<__half>(const __half *p)
{
    return (double)__half2float(*p);
}
template <> __device__ __forceinline__ double chk_d<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return (double)__bfloat162float(*p);
}

// The three sums of one plane into part[0..2].  p0: element offset of the
// plane's interior point (0, 0); sy, sz: row and plane strides (elements).
// Every thread of the block calls it.
template <class T, class CT>
__device__ __forceinline__ void check_plane_sums(const T *un, const T *up, const CT *cf,
                                                 int nx, int ny, long long p0, long long sy,
                                                 long long sz, double isu, double *part)
{
    const double c[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                         -1.0 / 560.0};
    double a0 = 0, a1 = 0, a2 = 0;
    for (int i = threadIdx.x; i < nx * ny; i += kCheckThreads) {
        const int x = i % nx, y = i / nx;
        const long long p = p0 + (long long)y * sy + x;
        const double u = chk_d(un + p) * isu;
        const double v = chk_d(up + p) * isu;
        double lap = 3.0 * c[0] * v;
        for (int m = 1; m <= 4; ++m)
            lap += c[m] * (chk_d(up + p - m) + chk_d(up + p + m) + chk_d(up + p - m * sy) +
                           chk_d(up + p + m * sy) + chk_d(up + p - m * sz) +
                           chk_d(up + p + m * sz)) * isu;
        const double d = u - v;
        a0 += u * u;
        a1 += d * d / chk_d(cf + p);
        a2 += u * lap;
    }
    __shared__ double red[3][kCheckThreads];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = kCheckThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[k] = red[k][0];
}

// nplanes triples of plane sums added in a fixed order into out[0..2]; one
// block of kCheckThreads threads.
__device__ __forceinline__ void check_sum_planes(const double *part, int nplanes, double *out)
{
    __shared__ double red[3][kCheckThreads];
    double a[3] = {0, 0, 0};
    for (int z = threadIdx.x; z < nplanes; z += kCheckThreads)
        for (int k = 0; k < 3; ++k) a[k] += part[3 * z + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = kCheckThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[k] = red[k][0];
}

}  // namespace gw
