// Host interface of the tcgen05 forward pass of the element-patch MLP (mlp_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace sisdc {

struct MlpTcArgs {
    const double* field;      // residual r, rows of q values (state layout)
    const float* sinv;        // per row: 1 / patch scale
    const float* s;           // per row: patch scale
    double* z;                // output z = r + s MLP(patch / s) (or z += ...)
    int add;
    const float *b1, *b2, *b3;
    int nex, ney, q, n_in, H;
    int nP1;                  // 64-wide K panels of layer 1: ceil(n_in / 64)
    int N3;                   // layer-3 width: q rounded up to 16
    long long rows;
    float feat;               // the scalar feature 0.1 log(c / h^2)
    int* err;                 // device flag: set when a wait timed out
};

// the forward pass fits the kernel (H a multiple of 16 up to 128, q <= 128,
// shared memory); *smem = dynamic shared memory bytes of the launch
bool mlp_tc_eligible(int n_in, int H, int q, size_t* smem);
// TMA descriptor of a [rows][cols] BF16 row-major matrix (cols % 64 == 0),
// boxes of 64 columns x box_rows rows, 128-byte swizzle; map = 128 bytes,
// 64-byte aligned
bool mlp_tc_encode(void* map, const void* ptr, int rows, int cols, int box_rows);
// the transposed, padded BF16 weights W1^T [H][K1p], W2^T [H][128], W3^T [N3][128]
cudaError_t mlp_tc_pack(const float* W1, const float* W2, const float* W3, int n_in, int H, int q, int K1p, int N3,
                        void* W1T, void* W2T, void* W3T, cudaStream_t s);
// one persistent launch over all rows (grid = min(tiles, nsm))
cudaError_t mlp_tc_forward(const MlpTcArgs& a, const void* m1, const void* m2, const void* m3, int nsm,
                           cudaStream_t s);

}  // namespace sisdc
