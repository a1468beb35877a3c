// pd_stencil_d3q4.cu -- the compile-time stencil step variants for a
// 3D grid with 4 parts of the half-stencil per row pair
// (one translation unit per pair, so that the build compiles them in parallel).
#include "pd_stencil_kernel.cuh"

namespace pdi {

StencilKernelFn stencil_pick_d3q4(int ns, int law, bool kappa, bool fo) {
    return pick_variant<3, 4>(ns, law, kappa, fo);
}

StencilPairFn stencil_pair_d3q4(int law, bool kappa) { return pick_pair_variant<3, 4>(law, kappa); }

}  // namespace pdi
