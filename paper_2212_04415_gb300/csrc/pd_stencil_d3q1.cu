// pd_stencil_d3q1.cu -- the compile-time stencil step variants for a
// 3D grid with 1 part of the half-stencil per row pair
// (one translation unit per pair, so that the build compiles them in parallel).
#include "pd_stencil_kernel.cuh"

namespace pdi {

StencilKernelFn stencil_pick_d3q1(int ns, int law, bool kappa, bool fo) {
    return pick_variant<3, 1>(ns, law, kappa, fo);
}

StencilPairFn stencil_pair_d3q1(int law, bool kappa) { return pick_pair_variant<3, 1>(law, kappa); }

}  // namespace pdi
