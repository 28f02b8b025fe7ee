// Dispatch of the persistent sweep kernel by PDE, degree and precision.
#include "ops.h"

namespace sisdc {

int sweep_config_pde0_lo_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_lo_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde0_hi_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_hi_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde0_lo_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_lo_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde0_hi_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_hi_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_lo_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_lo_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_hi_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_hi_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_lo_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_lo_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde1_hi_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde1_hi_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_lo_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_lo_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_hi_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_hi_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_lo_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_lo_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde2_hi_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde2_hi_1(const SweepArgs& a, int grid, int block);

int sweep_config_pde3_lo_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde3_lo_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde3_hi_0(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde3_hi_0(const SweepArgs& a, int grid, int block);
int sweep_config_pde3_lo_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde3_lo_1(const SweepArgs& a, int grid, int block);
int sweep_config_pde3_hi_1(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde3_hi_1(const SweepArgs& a, int grid, int block);

int sweep_config_pde0_1dhi(const Geo& g, int* epb, int* block);
cudaError_t sweep_launch_pde0_1dhi(const SweepArgs& a, int grid, int block);

int sweep_config(const Geo& g, int pde, int mix, int* epb, int* block) {
    if (g.nq > 9) return pde == 0 && !mix ? sweep_config_pde0_1dhi(g, epb, block) : 0;
    const bool lo = g.nq < 6;
    mix = mix ? 1 : 0;
    if (pde == 0 && mix == 0) return lo ? sweep_config_pde0_lo_0(g, epb, block) : sweep_config_pde0_hi_0(g, epb, block);
    if (pde == 0 && mix == 1) return lo ? sweep_config_pde0_lo_1(g, epb, block) : sweep_config_pde0_hi_1(g, epb, block);
    if (pde == 1 && mix == 0) return lo ? sweep_config_pde1_lo_0(g, epb, block) : sweep_config_pde1_hi_0(g, epb, block);
    if (pde == 1 && mix == 1) return lo ? sweep_config_pde1_lo_1(g, epb, block) : sweep_config_pde1_hi_1(g, epb, block);
    if (pde == 2 && mix == 0) return lo ? sweep_config_pde2_lo_0(g, epb, block) : sweep_config_pde2_hi_0(g, epb, block);
    if (pde == 2 && mix == 1) return lo ? sweep_config_pde2_lo_1(g, epb, block) : sweep_config_pde2_hi_1(g, epb, block);
    if (pde == 3 && mix == 0) return lo ? sweep_config_pde3_lo_0(g, epb, block) : sweep_config_pde3_hi_0(g, epb, block);
    if (pde == 3 && mix == 1) return lo ? sweep_config_pde3_lo_1(g, epb, block) : sweep_config_pde3_hi_1(g, epb, block);
    return 0;
}

cudaError_t launch_sweep(const SweepArgs& a, int grid, int block) {
    if (a.g.nq > 9) return a.pde == 0 && !a.mix ? sweep_launch_pde0_1dhi(a, grid, block) : cudaErrorInvalidValue;
    const bool lo = a.g.nq < 6;
    const int mix = a.mix ? 1 : 0;
    if (a.pde == 0 && mix == 0) return lo ? sweep_launch_pde0_lo_0(a, grid, block) : sweep_launch_pde0_hi_0(a, grid, block);
    if (a.pde == 0 && mix == 1) return lo ? sweep_launch_pde0_lo_1(a, grid, block) : sweep_launch_pde0_hi_1(a, grid, block);
    if (a.pde == 1 && mix == 0) return lo ? sweep_launch_pde1_lo_0(a, grid, block) : sweep_launch_pde1_hi_0(a, grid, block);
    if (a.pde == 1 && mix == 1) return lo ? sweep_launch_pde1_lo_1(a, grid, block) : sweep_launch_pde1_hi_1(a, grid, block);
    if (a.pde == 2 && mix == 0) return lo ? sweep_launch_pde2_lo_0(a, grid, block) : sweep_launch_pde2_hi_0(a, grid, block);
    if (a.pde == 2 && mix == 1) return lo ? sweep_launch_pde2_lo_1(a, grid, block) : sweep_launch_pde2_hi_1(a, grid, block);
    if (a.pde == 3 && mix == 0) return lo ? sweep_launch_pde3_lo_0(a, grid, block) : sweep_launch_pde3_hi_0(a, grid, block);
    if (a.pde == 3 && mix == 1) return lo ? sweep_launch_pde3_lo_1(a, grid, block) : sweep_launch_pde3_hi_1(a, grid, block);
    return cudaErrorInvalidValue;
}

}  // namespace sisdc
