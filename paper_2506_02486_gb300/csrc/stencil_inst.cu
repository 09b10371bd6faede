// stencil_inst.cu -- one tile configuration of the fused step kernel per
// object file.  The build compiles this file once per configuration with
// -DGW_INST=<index> so that the instantiations compile in parallel; the
// index -> (storage type, tile) table is mirrored in stencil_dispatch.cpp.
#include "stencil.cuh"

#ifndef GW_INST
#error "compile with -DGW_INST=<configuration index>"
#endif

namespace gw {

// Cfg<storage, tile x, tile y, rows per thread, u-ring slots, pointwise
//     slots, CTAs per SM wanted, packed f32x2 math, planes per queue shift>
#if GW_INST == 0
using C = Cfg<float, 64, 28, 2, 8, 4>;  constexpr bool kDelta = false;
#elif GW_INST == 1
using C = Cfg<float, 128, 14, 2, 8, 4>; constexpr bool kDelta = false;
#elif GW_INST == 2
using C = Cfg<float, 32, 56, 2, 8, 4>;  constexpr bool kDelta = false;
#elif GW_INST == 3
using C = Cfg<float, 64, 28, 2, 10, 5>; constexpr bool kDelta = false;
#elif GW_INST == 4
using C = Cfg<double, 32, 16, 1, 7, 3>; constexpr bool kDelta = false;
#elif GW_INST == 5
using C = Cfg<double, 64, 8, 1, 7, 3>;  constexpr bool kDelta = false;
#elif GW_INST == 6
using C = Cfg<__half, 64, 28, 2, 8, 4>;  constexpr bool kDelta = true;
#elif GW_INST == 7
using C = Cfg<__half, 128, 14, 2, 8, 4>; constexpr bool kDelta = true;
#elif GW_INST == 8
using C = Cfg<__half, 64, 28, 2, 12, 6>; constexpr bool kDelta = true;
#elif GW_INST == 9
using C = Cfg<__nv_bfloat16, 64, 28, 2, 8, 4>;  constexpr bool kDelta = true;
#elif GW_INST == 10
using C = Cfg<__nv_bfloat16, 128, 14, 2, 8, 4>; constexpr bool kDelta = true;
#elif GW_INST == 11
using C = Cfg<__nv_bfloat16, 64, 28, 2, 12, 6>; constexpr bool kDelta = true;
#elif GW_INST == 12
using C = Cfg<float, 64, 28, 2, 8, 4, 1, false>;  constexpr bool kDelta = false;
#elif GW_INST == 13
using C = Cfg<float, 64, 14, 1, 8, 4, 2, true>;   constexpr bool kDelta = false;
#elif GW_INST == 14
using C = Cfg<float, 128, 7, 1, 8, 4, 2, true>;   constexpr bool kDelta = false;
#elif GW_INST == 15
using C = Cfg<__half, 64, 14, 1, 8, 4, 2, true>;  constexpr bool kDelta = true;
#elif GW_INST == 16
using C = Cfg<__half, 32, 56, 2, 8, 4>;           constexpr bool kDelta = true;
#elif GW_INST == 17
using C = Cfg<__nv_bfloat16, 32, 56, 2, 8, 4>;    constexpr bool kDelta = true;
#else
#error "unknown configuration index"
#endif

#define GW_CAT2(a, b) a##b
#define GW_CAT(a, b) GW_CAT2(a, b)

cudaError_t GW_CAT(step_launch_, GW_INST)(bool sponge, int grid,
                                          const StepArgs &a, cudaStream_t s)
{
    return launch_cfg<C, kDelta>(sponge, grid, a, s);
}
int GW_CAT(step_occ_, GW_INST)(bool sponge) { return occ_cfg<C, kDelta>(sponge); }
TileInfo GW_CAT(step_info_, GW_INST)() { return info_of<C>(); }

}  // namespace gw
