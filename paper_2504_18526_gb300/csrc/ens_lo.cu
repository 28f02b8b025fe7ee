// Instantiations of the ensemble sweep kernel (NQ 2 3 4 5, FP64).
#include "ens.cuh"

namespace sisdc {

int ens_occupancy_lo(int nq, int epb) {
    switch (nq) {
        case 2: return ens_occupancy_impl<2, false>(epb);
        case 3: return ens_occupancy_impl<3, false>(epb);
        case 4: return ens_occupancy_impl<4, false>(epb);
        case 5: return ens_occupancy_impl<5, false>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_lo(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 2: return ens_launch_impl<2, false>(a, grid, s);
        case 3: return ens_launch_impl<3, false>(a, grid, s);
        case 4: return ens_launch_impl<4, false>(a, grid, s);
        case 5: return ens_launch_impl<5, false>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

// the same with at most 64 registers per thread (two 512-thread blocks per SM)
int ens_occupancy_lo2(int nq, int epb) {
    switch (nq) {
        case 2: return ens_occupancy_impl<2, false, 2>(epb);
        case 3: return ens_occupancy_impl<3, false, 2>(epb);
        case 4: return ens_occupancy_impl<4, false, 2>(epb);
        case 5: return ens_occupancy_impl<5, false, 2>(epb);
        default: return 0;
    }
}

cudaError_t ens_launch_lo2(const EnsArgs& a, int nq, int grid, cudaStream_t s) {
    switch (nq) {
        case 2: return ens_launch_impl<2, false, 2>(a, grid, s);
        case 3: return ens_launch_impl<3, false, 2>(a, grid, s);
        case 4: return ens_launch_impl<4, false, 2>(a, grid, s);
        case 5: return ens_launch_impl<5, false, 2>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
