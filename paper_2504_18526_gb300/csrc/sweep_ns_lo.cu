// Instantiations of the persistent sweep kernel (PDE 3 (Navier-Stokes), NQ 2..5, FP64).
#include "sweep.cuh"

namespace sisdc {

int sweep_config_pde3_lo_0(const Geo& g, int* epb, int* block) {
    switch (g.nq * 10 + g.dim) {
        case 22: return sweep_config_impl<2, 2, 3, false>(g, epb, block);
        case 32: return sweep_config_impl<3, 2, 3, false>(g, epb, block);
        case 42: return sweep_config_impl<4, 2, 3, false>(g, epb, block);
        case 52: return sweep_config_impl<5, 2, 3, false>(g, epb, block);
        default: return 0;
    }
}

cudaError_t sweep_launch_pde3_lo_0(const SweepArgs& a, int grid, int block) {
    switch (a.g.nq * 10 + a.g.dim) {
        case 22: return sweep_launch_impl<2, 2, 3, false>(a, grid, block);
        case 32: return sweep_launch_impl<3, 2, 3, false>(a, grid, block);
        case 42: return sweep_launch_impl<4, 2, 3, false>(a, grid, block);
        case 52: return sweep_launch_impl<5, 2, 3, false>(a, grid, block);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
