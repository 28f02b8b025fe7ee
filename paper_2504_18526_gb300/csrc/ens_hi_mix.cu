// Instantiations of the ensemble sweep kernel (NQ 6 7 8 9, mixed precision).
#include "ens.cuh"

namespace sisdc {

int ens_occupancy_hi_mix(int nq, int epb) {
    switch (nq) {
        case 6: return ens_occupancy_impl<6, true>(epb);
        case 7: return ens_occupancy_impl<7, true>(epb);
        case 8: return ens_occupancy_impl<8, true>(epb);
        case 9: return ens_occupancy_impl<9, true>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_hi_mix(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 6: return ens_launch_impl<6, true>(a, grid, s);
        case 7: return ens_launch_impl<7, true>(a, grid, s);
        case 8: return ens_launch_impl<8, true>(a, grid, s);
        case 9: return ens_launch_impl<9, true>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

// the same with at most 64 registers per thread (two 512-thread blocks per SM)
int ens_occupancy_hi_mix2(int nq, int epb) {
    switch (nq) {
        case 6: return ens_occupancy_impl<6, true, 2>(epb);
        case 7: return ens_occupancy_impl<7, true, 2>(epb);
        case 8: return ens_occupancy_impl<8, true, 2>(epb);
        case 9: return ens_occupancy_impl<9, true, 2>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_hi_mix2(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 6: return ens_launch_impl<6, true, 2>(a, grid, s);
        case 7: return ens_launch_impl<7, true, 2>(a, grid, s);
        case 8: return ens_launch_impl<8, true, 2>(a, grid, s);
        case 9: return ens_launch_impl<9, true, 2>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
