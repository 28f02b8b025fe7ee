// Instantiations of the ensemble sweep kernel (NQ 4 5, mixed precision).
#include "ens.cuh"

namespace sisdc {

int ens_occupancy_lo_mix(int nq, int epb) {
    switch (nq) {
        case 4: return ens_occupancy_impl<4, true>(epb);
        case 5: return ens_occupancy_impl<5, true>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_lo_mix(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 4: return ens_launch_impl<4, true>(a, grid, s);
        case 5: return ens_launch_impl<5, true>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

// the same with at most 64 registers per thread (two 512-thread blocks per SM)
int ens_occupancy_lo_mix2(int nq, int epb) {
    switch (nq) {
        case 4: return ens_occupancy_impl<4, true, 2>(epb);
        case 5: return ens_occupancy_impl<5, true, 2>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_lo_mix2(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 4: return ens_launch_impl<4, true, 2>(a, grid, s);
        case 5: return ens_launch_impl<5, true, 2>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
