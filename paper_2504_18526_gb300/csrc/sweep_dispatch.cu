// Dispatch of the persistent sweep kernel by PDE and degree.
#include "ops.h"

namespace sisdc {

int sweep_config_pde0_lo(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_lo(const SweepArgs& a, int grid, int block);
int sweep_config_pde0_hi(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_hi(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_lo(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_lo(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_hi(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_hi(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_lo(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_lo(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_hi(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_hi(const SweepArgs& a, int grid, int block);

int sweep_config(const Geo& g, int pde, int* epb, int* block) {
    const bool lo = g.nq < 6;
    switch (pde) {
        case 0: return lo ? sweep_config_pde0_lo(g, epb, block) : sweep_config_pde0_hi(g, epb, block);
        case 1: return lo ? sweep_config_pde1_lo(g, epb, block) : sweep_config_pde1_hi(g, epb, block);
        case 2: return lo ? sweep_config_pde2_lo(g, epb, block) : sweep_config_pde2_hi(g, epb, block);
        default: return 0;
    }
}

cudaError_t launch_sweep(const SweepArgs& a, int grid, int block) {
    const bool lo = a.g.nq < 6;
    switch (a.pde) {
        case 0: return lo ? sweep_launch_pde0_lo(a, grid, block) : sweep_launch_pde0_hi(a, grid, block);
        case 1: return lo ? sweep_launch_pde1_lo(a, grid, block) : sweep_launch_pde1_hi(a, grid, block);
        case 2: return lo ? sweep_launch_pde2_lo(a, grid, block) : sweep_launch_pde2_hi(a, grid, block);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
