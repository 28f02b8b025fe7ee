// Instantiations of the persistent sweep kernel for 1D convection-diffusion
// levels of degree 9..15 (NQ 10..16, FP64).
#include "sweep.cuh"

namespace sisdc {

int sweep_config_pde0_1dhi(const Geo& g, int* epb, int* block) {
    if (g.dim != 1) return 0;
    switch (g.nq) {
        case 10: return sweep_config_impl<10, 1, 0, false>(g, epb, block);
        case 11: return sweep_config_impl<11, 1, 0, false>(g, epb, block);
        case 12: return sweep_config_impl<12, 1, 0, false>(g, epb, block);
        case 13: return sweep_config_impl<13, 1, 0, false>(g, epb, block);
        case 14: return sweep_config_impl<14, 1, 0, false>(g, epb, block);
        case 15: return sweep_config_impl<15, 1, 0, false>(g, epb, block);
        case 16: return sweep_config_impl<16, 1, 0, false>(g, epb, block);
        default: return 0;
    }
}

cudaError_t sweep_launch_pde0_1dhi(const SweepArgs& a, int grid, int block) {
    if (a.g.dim != 1) return cudaErrorInvalidValue;
    switch (a.g.nq) {
        case 10: return sweep_launch_impl<10, 1, 0, false>(a, grid, block);
        case 11: return sweep_launch_impl<11, 1, 0, false>(a, grid, block);
        case 12: return sweep_launch_impl<12, 1, 0, false>(a, grid, block);
        case 13: return sweep_launch_impl<13, 1, 0, false>(a, grid, block);
        case 14: return sweep_launch_impl<14, 1, 0, false>(a, grid, block);
        case 15: return sweep_launch_impl<15, 1, 0, false>(a, grid, block);
        case 16: return sweep_launch_impl<16, 1, 0, false>(a, grid, block);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
