// Instantiations of the persistent sweep kernel (PDE 3 (Navier-Stokes), NQ 6..9, FP64).
#include "sweep.cuh"

namespace sisdc {

int sweep_config_pde3_hi_0(const Geo& g, int* epb, int* block) {
    switch (g.nq * 10 + g.dim) {
        case 62: return sweep_config_impl<6, 2, 3, false>(g, epb, block);
        case 72: return sweep_config_impl<7, 2, 3, false>(g, epb, block);
        case 82: return sweep_config_impl<8, 2, 3, false>(g, epb, block);
        case 92: return sweep_config_impl<9, 2, 3, false>(g, epb, block);
        default: return 0;
    }
}

cudaError_t sweep_launch_pde3_hi_0(const SweepArgs& a, int grid, int block) {
    switch (a.g.nq * 10 + a.g.dim) {
        case 62: return sweep_launch_impl<6, 2, 3, false>(a, grid, block);
        case 72: return sweep_launch_impl<7, 2, 3, false>(a, grid, block);
        case 82: return sweep_launch_impl<8, 2, 3, false>(a, grid, block);
        case 92: return sweep_launch_impl<9, 2, 3, false>(a, grid, block);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
