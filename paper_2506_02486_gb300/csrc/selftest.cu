// selftest.cu -- gw_selftest_timeout: makes the two kinds of device wait
// the step kernel uses run out, on purpose and harmlessly, so that a test
// can check that a wait which never completes ends with an error status the
// host reads while the context stays usable.
//
// One warp: lane 0 waits on a shared-memory mbarrier that nobody arrives
// on, then on a global counter that nobody increments, each bounded by the
// caller's limit (the step kernel bounds the same waits by kWaitLimitNs).
// Each wait that gives up sets a bit of the result word.
#include <cuda_runtime.h>

#include "gw_internal.h"
#include "ptx.cuh"

namespace gw {
namespace {

__device__ unsigned g_selftest_counter;   // never incremented
__device__ unsigned g_selftest_result;

__global__ void k_selftest_timeout(unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    unsigned bits = 0;
    mbar_init(&bar, 1);
    fence_barrier_init();
    // (1) an mbarrier phase that never completes
    {
        const unsigned long long t0 = global_timer();
        for (uint32_t i = 0;; ++i) {
            if (mbar_try_wait(&bar, 0)) break;
            if ((i & 63u) == 63u && global_timer() - t0 > limit_ns) {
                bits |= 1u;
                break;
            }
        }
    }
    // (2) a device-wide counter that never reaches its target
    {
        const unsigned long long t0 = global_timer();
        for (uint32_t i = 0;; ++i) {
            if (ld_acquire_gpu(&g_selftest_counter) >= 1u) break;
            if ((i & 63u) == 63u && global_timer() - t0 > limit_ns) {
                bits |= 2u;
                break;
            }
        }
    }
    g_selftest_result = bits;
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" gw_status gw_selftest_timeout(gw_ctx *c, unsigned limit_us, int *expired)
{
    if (!c || !expired) return fail(GW_ERR_ARG, "NULL argument");
    if (c->device < 0) return fail(GW_ERR_STATE, "the self-test needs a device context");
    if (limit_us == 0 || limit_us > 2000000u)
        return fail(GW_ERR_ARG, "limit must be 1 us .. 2 s");
    GW_TRY_CUDA(cudaSetDevice(c->device));
    const unsigned zero = 0;
    GW_TRY_CUDA(cudaMemcpyToSymbol(g_selftest_counter, &zero, sizeof zero));
    GW_TRY_CUDA(cudaMemcpyToSymbol(g_selftest_result, &zero, sizeof zero));
    k_selftest_timeout<<<1, 32>>>((unsigned long long)limit_us * 1000ull);
    GW_TRY_CUDA(cudaGetLastError());
    GW_TRY_CUDA(cudaStreamSynchronize(nullptr));
    unsigned bits = 0;
    GW_TRY_CUDA(cudaMemcpyFromSymbol(&bits, g_selftest_result, sizeof bits));
    *expired = (int)bits;
    if (bits) return fail(GW_ERR_TIMEOUT, "device waits gave up as intended (bits 0x%x)", bits);
    return GW_OK;
}
