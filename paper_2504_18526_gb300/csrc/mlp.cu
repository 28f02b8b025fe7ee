// Element-patch MLP for the implicit stage: inference, training, learned solve.
//
// Not in the paper (a learned initial guess / preconditioner for the implicit
// equations of Sec. 3.3).  For every element and component the 3x3 element
// patch of a nodal residual field r (9 Q values, neighbour offsets (dy, dx)
// in {-1,0,1}^2 row-major) is scaled by its RMS s and extended by the
// feature 0.1 log(c / h^2); a perceptron n_in -> H -> H -> Q with tanh hidden
// layers predicts the deviation of the centre element's correction from r
// itself (the exact correction as c -> 0): z = r + s MLP(r_patch / s).
// BF16 mode (the default): weights are BF16 (FP32 master copy for training),
// both operands of every GEMM are BF16 on the tensor cores (warp-level
// mma.sync m16n8k16) with FP32 accumulation, and the patch matrix is stored
// in BF16.  FP32 mode: the same network with FP32 SIMT GEMMs, the reference
// form for the gradient checks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sisdc.h"
#include "ds.cuh"
#include "mlp_tc.h"
#include "ops.h"

namespace sisdc {

// ---- kernels ---------------------------------------------------------------

// patch gathering in three elementwise passes (rows = element-components):
// sum of squares of each row's q values; the patch scale s = RMS over the 3x3
// patch from the nine neighbours' sums; then every input X[row][t] (the
// patch values scaled by 1/s, and the feature) by one thread
__global__ void k_mlp_elem_ss(const double* __restrict__ f, long long rows, int q, double* __restrict__ ss) {
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long long)gridDim.x * blockDim.x) {
        const double* v = f + row * q;
        double a = 0.0;
        for (int k = 0; k < q; ++k) a += v[k] * v[k];
        ss[row] = a;
    }
}

__global__ void k_mlp_scale(const double* __restrict__ ss, int nex, int ney, int q, long long rows,
                            float* __restrict__ s, float* __restrict__ sinv) {
    const int nel = nex * ney;
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(row / nel), e = (int)(row - (long long)c * nel);
        const int ex = e % nex, ey = e / nex;
        double tot = 0.0;
        for (int k = 0; k < 9; ++k) {
            const int dy = k / 3 - 1, dx = k % 3 - 1;
            tot += ss[(long long)c * nel + ((ey + dy + ney) % ney) * nex + (ex + dx + nex) % nex];
        }
        double sc = sqrt(tot / (9.0 * q));
        sc = sc > 0.0 ? sc : 1.0;
        s[row] = (float)sc;
        sinv[row] = (float)(1.0 / sc);
    }
}

// (FP32 arithmetic: the value rounded to FP32 on the integer pipe, then
// scaled; GB300's FP64 unit would otherwise set this kernel's time).  A thread
// keeps the same input slots t = threadIdx.x + j blockDim.x for every row, so
// their (neighbour, node) split is computed once; the nine neighbour offsets
// of a row are computed once per row in shared memory.
constexpr int FILL_THREADS = 128, FILL_SLOTS = 8;   // n_in <= 1024

template <class TX>
__device__ __forceinline__ TX to_x(float v);
template <>
__device__ __forceinline__ float to_x<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_x<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// X[row][t] for t < n_in, rows ldx apart (FP32, or BF16 for the tensor cores)
template <class TX>
__global__ void __launch_bounds__(FILL_THREADS) k_mlp_fill(const double* __restrict__ f, const float* __restrict__ sinv,
                                                         int nex, int ney, int q, long long rows, int n_in, int ldx,
                                                         float feat, TX* __restrict__ X) {
    __shared__ long long nbase[9];
    const int nel = nex * ney;
    const long long N = (long long)nel * q;
    int tk[FILL_SLOTS], tn[FILL_SLOTS];
#pragma unroll
    for (int j = 0; j < FILL_SLOTS; ++j) {
        const int t = threadIdx.x + j * FILL_THREADS;
        tk[j] = t / q;
        tn[j] = t - tk[j] * q;
    }
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        if (threadIdx.x < 9) {
            const int c = (int)(row / nel), e = (int)(row - (long long)c * nel);
            const int ex = e % nex, ey = e / nex;
            const int dy = (int)threadIdx.x / 3 - 1, dx = (int)threadIdx.x % 3 - 1;
            nbase[threadIdx.x] = c * N + (long long)(((ey + dy + ney) % ney) * nex + (ex + dx + nex) % nex) * q;
        }
        __syncthreads();
        const float si = sinv[row];
        TX* xr = X + row * ldx;
#pragma unroll
        for (int j = 0; j < FILL_SLOTS; ++j) {
            const int t = threadIdx.x + j * FILL_THREADS;
            if (t < 9 * q) xr[t] = to_x<TX>(d2f_int(f[nbase[tk[j]] + tn[j]]) * si);
            else if (t == 9 * q) xr[t] = to_x<TX>(feat);
        }
        __syncthreads();
    }
}

// targets t = (dx - r_centre) / s
__global__ void k_mlp_targets(const double* __restrict__ dx, const double* __restrict__ r, const float* __restrict__ s,
                              int q, long long rows, float* __restrict__ T) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < rows * q; k += (long long)gridDim.x * blockDim.x) {
        const long long row = k / q;
        T[k] = d2f_int(dx[k] - r[k]) / s[row];
    }
}

// z (+)= r_centre + s * y (state layout = row-major rows of q values)
__global__ void k_mlp_scatter(const float* __restrict__ Y, const float* __restrict__ s, const double* __restrict__ r,
                              int q, long long rows, double* __restrict__ z, int add) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < rows * q; k += (long long)gridDim.x * blockDim.x) {
        const double v = r[k] + f2d_int(Y[k] * s[k / q]);
        z[k] = add ? z[k] + v : v;
    }
}

template <class T>
__device__ __forceinline__ float ld_as_float(const T* p, long long i);
template <>
__device__ __forceinline__ float ld_as_float<float>(const float* p, long long i) { return p[i]; }
template <>
__device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(p[i]);
}

// C[MxN] = op(A) op(B) (+ bias) (tanh), FP32 accumulation; A element (m,k)
// at A[m*lda + k] (or A[k*lda + m] when ta), B element (k,n) at B[k*ldb + n]
// (or B[n*ldb + k] when tb).  64x64 tiles, 16-wide K slices, 4x4 per thread.
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_TANH = 2 };

template <class TA, class TB>
__global__ void k_gemm(const TA* __restrict__ A, const TB* __restrict__ B, float* __restrict__ C, const float* bias,
                       int M, int N, int K, int lda, int ldb, int ldc, int ta, int tb, int epi) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, mm = t % 64;
            const int m = m0 + mm, k = k0 + kk;
            float va = 0.f;
            if (m < M && k < K) va = ld_as_float<TA>(A, ta ? (long long)k * lda + m : (long long)m * lda + k);
            As[kk][mm] = va;
            const int n = n0 + mm;
            float vb = 0.f;
            if (n < N && k < K) vb = ld_as_float<TB>(B, tb ? (long long)n * ldb + k : (long long)k * ldb + n);
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = Bs[kk][tx * 4 + r];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = m0 + ty * 4 + r, n = n0 + tx * 4 + q;
            if (m < M && n < N) {
                float v = acc[r][q];
                if (epi >= EPI_BIAS) v += bias[n];
                if (epi == EPI_BIAS_TANH) v = tanhf(v);
                C[(long long)m * ldc + n] = v;
            }
        }
}

// Tensor-core form of k_gemm for the BF16 mode: both operands are rounded to
// BF16 while they are staged in shared memory and multiplied by warp-level
// mma.sync m16n8k16 (BF16 x BF16 -> FP32 accumulate).  Block tile 64x64,
// K slices of 32, 4 warps each owning a 32x32 sub-tile (2 x 4 MMA tiles).
// kz > 1 (split-K): block z covers K slices [z * kchunk, (z+1) * kchunk) and
// writes its partial product to C + z * M * N (row-major M x N, no epilogue);
// k_splitk_sum adds the partials in a fixed order.
constexpr int TC_BM = 64, TC_BN = 64, TC_BK = 32, TC_PAD = 8;

__device__ __forceinline__ void mma_bf16_16816(float* d, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <class TA, class TB, bool ta, bool tb>
__global__ void __launch_bounds__(128, 4) k_gemm_tc(const TA* __restrict__ A, const TB* __restrict__ B,
                                                 float* __restrict__ C, const float* bias, int M, int N, int K,
                                                 int lda, int ldb, int ldc, int epi, int kchunk) {
    __shared__ __align__(16) __nv_bfloat16 As[TC_BM][TC_BK + TC_PAD];   // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[TC_BN][TC_BK + TC_PAD];   // [n][k]
    constexpr int PER = TC_BM * TC_BK / 128;                           // staged elements per thread and operand
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    // staging slot i of this thread: consecutive threads walk the operand's
    // contiguous index (k for row-major A, m for transposed A; n / k for B)
    auto slotA = [&](int i, int& mm, int& kk) {
        const int t = threadIdx.x + i * 128;
        if constexpr (ta) { kk = t / TC_BM; mm = t - kk * TC_BM; } else { mm = t / TC_BK; kk = t - mm * TC_BK; }
    };
    auto slotB = [&](int i, int& nn, int& kk) {
        const int t = threadIdx.x + i * 128;
        if constexpr (tb) { nn = t / TC_BK; kk = t - nn * TC_BK; } else { kk = t / TC_BN; nn = t - kk * TC_BN; }
    };
    // a row-major BF16 A (rows 16-byte aligned: lda % 8 == 0, checked by the
    // host) is staged 8 values per 16-byte load
    constexpr bool VA = std::is_same<TA, __nv_bfloat16>::value && !ta;
    constexpr int PA = VA ? TC_BM * TC_BK / 8 / 128 : PER;             // staged A items per thread
    float ra[VA ? 1 : PER], rb[PER];
    uint4 va[VA ? PA : 1];
    auto slotV = [&](int i, int& mm, int& kq) {
        const int c = threadIdx.x + i * 128;
        mm = c / (TC_BK / 8);
        kq = (c - mm * (TC_BK / 8)) * 8;
    };
    // global -> registers for the slice at k0 (all loads issued before use)
    auto fetch = [&](int k0) {
        if constexpr (VA) {
#pragma unroll
            for (int i = 0; i < PA; ++i) {
                int mm, kq;
                slotV(i, mm, kq);
                const int m = m0 + mm, k = k0 + kq;
                if (m < M && k + 8 <= kend) {
                    va[i] = *reinterpret_cast<const uint4*>(A + (long long)m * lda + k);
                } else {
                    __align__(16) __nv_bfloat16 tmp[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        tmp[e] = (m < M && k + e < kend) ? A[(long long)m * lda + k + e] : __float2bfloat16_rn(0.f);
                    va[i] = *reinterpret_cast<const uint4*>(tmp);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if constexpr (!VA) {
                int mm, kk;
                slotA(i, mm, kk);
                const int m = m0 + mm, k = k0 + kk;
                ra[i] = (m < M && k < kend) ? ld_as_float<TA>(A, ta ? (long long)k * lda + m : (long long)m * lda + k) : 0.f;
            }
            int nn, kb;
            slotB(i, nn, kb);
            const int n = n0 + nn, kq = k0 + kb;
            rb[i] = (n < N && kq < kend) ? ld_as_float<TB>(B, tb ? (long long)n * ldb + kq : (long long)kq * ldb + n) : 0.f;
        }
    };
    float acc[2][4][4] = {};
    if (kbeg < kend) fetch(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += TC_BK) {
        if constexpr (VA) {
#pragma unroll
            for (int i = 0; i < PA; ++i) {
                int mm, kq;
                slotV(i, mm, kq);
                *reinterpret_cast<uint4*>(&As[mm][kq]) = va[i];
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if constexpr (!VA) {
                int mm, kk;
                slotA(i, mm, kk);
                As[mm][kk] = __float2bfloat16_rn(ra[i]);
            }
            int nn, kb;
            slotB(i, nn, kb);
            Bs[nn][kb] = __float2bfloat16_rn(rb[i]);
        }
        __syncthreads();
        if (k0 + TC_BK < kend) fetch(k0 + TC_BK);     // next slice in flight during the MMAs
#pragma unroll
        for (int kk = 0; kk < TC_BK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * t4]);
                af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * t4]);
                af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * t4 + 8]);
                af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bfr[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * t4]);
                bfr[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    float* Cz = gridDim.z > 1 ? C + (size_t)blockIdx.z * M * N : C;
    const int ldz = gridDim.z > 1 ? N : ldc;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + i * 16 + g + (h >> 1) * 8;
                const int n = n0 + wn + j * 8 + 2 * t4 + (h & 1);
                if (m < M && n < N) {
                    float v = acc[i][j][h];
                    if (gridDim.z == 1) {
                        if (epi >= EPI_BIAS) v += bias[n];
                        if (epi == EPI_BIAS_TANH) v = tanhf(v);
                    }
                    Cz[(long long)m * ldz + n] = v;
                }
            }
}

// C[m][n] = sum over z of the split-K partials P[z][m][n] (fixed order)
__global__ void k_splitk_sum(const float* __restrict__ P, int nz, int M, int N, float* __restrict__ C, int ldc) {
    const long long mn = (long long)M * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < mn; t += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < nz; ++z) v += P[z * mn + t];
        C[(t / N) * ldc + t % N] = v;
    }
}

// dY = (Y - T) / (rows * q); loss partials
__global__ void k_mlp_loss(const float* __restrict__ Y, const float* __restrict__ T, long long n, float scale,
                           float* __restrict__ dY, double* __restrict__ partial) {
    __shared__ double scratch[32];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float d = Y[k] - T[k];
        dY[k] = d * scale;
        acc += (double)d * (double)d;
    }
    const double s = block_sum(acc, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// *acc += scale * (sum of the n partials, in order)
__global__ void k_loss_acc(const double* __restrict__ partial, int n, double scale, double* __restrict__ acc) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += partial[b];
        *acc += scale * s;
    }
}

// dH *= (1 - H^2) (tanh derivative)
__global__ void k_tanh_back(const float* __restrict__ H, float* __restrict__ dH, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dH[k] *= 1.f - H[k] * H[k];
}

// column sums (bias gradients), one thread per column, fixed order
// column sums of D[rows][cols] in two deterministic passes: block (x, y)
// sums rows [y*chunk, (y+1)*chunk) of 32 columns with 8 row lanes (coalesced
// 32-column rows), partial[y][col]; then out[col] = sum over y in order
constexpr int COLSUM_CHUNKS = 64;

__global__ void k_colsum_part(const float* __restrict__ D, int rows, int cols, int chunk, float* __restrict__ part) {
    __shared__ float sh[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.f;
    if (c < cols)
        for (int i = r0 + threadIdx.y; i < r1; i += 8) s += D[(long long)i * cols + c];
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += sh[k][threadIdx.x];
        part[(long long)blockIdx.y * cols + c] = t;
    }
}

__global__ void k_colsum_fin(const float* __restrict__ part, int nchunk, int cols, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[(long long)k * cols + c];
    out[c] = s;
}

// Adam step on FP32 master weights; refresh the BF16 copy
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        wb[k] = __float2bfloat16(w[k]);
    }
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        wb[k] = __float2bfloat16(w[k]);
}

static unsigned ew(long long n) {
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace sisdc

using namespace sisdc;

struct sisdc_mlp_s {
    sisdc_level lvl = nullptr;
    int nc = 0, nex = 0, ney = 0, q = 0, n_in = 0, H = 0, bf16 = 1;
    long long rows = 0, nparam = 0;
    double h = 1.0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* theta_b = nullptr;
    float *X = nullptr, *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *T = nullptr, *dY = nullptr, *dH = nullptr,
          *s = nullptr;
    double* part = nullptr;
    float* ws = nullptr;            // split-K partials of the tensor-core GEMMs
    __nv_bfloat16* Xb = nullptr;    // BF16 mode: the patch inputs, rows ldx apart (zero padding)
    int ldx = 0;
    double* ss = nullptr;                    // per-row sums of squares
    float* sinv = nullptr;                   // 1 / patch scale
    double* lacc = nullptr;                  // loss accumulator of a training epoch
    long long adam_t = 0;
    // tcgen05 forward pass (mlp_tc.cu): transposed BF16 weights, their TMA
    // descriptors, and whether it is available / selected
    __nv_bfloat16 *W1T = nullptr, *W2T = nullptr, *W3T = nullptr;
    alignas(64) unsigned char tmap[3][128];
    int tc_ok = 0, use_tc = 1, K1p = 0, N3 = 0, nsm = 0;
    int* derr = nullptr;
    std::string err;
    // offsets
    long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

struct MlpFail {
    sisdc_status st;
};

void mck(sisdc_mlp_s* p, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        p->err = std::string(what) + ": " + cudaGetErrorString(e);
        throw MlpFail{SISDC_E_CUDA};
    }
}

// split-K workspace limit (floats)
constexpr long long MLP_SPLITK_WS = 1ll << 22;

// C = op(A) op(B) (+ bias, tanh): tensor cores in the BF16 mode (split-K when
// the output has too few tiles for the GPU and K is long, as for the weight
// gradients whose reduction runs over all rows), FP32 SIMT otherwise
template <class TB, class TA = float>
void gemm(sisdc_mlp_s* p, const TA* A, const TB* B, float* C, const float* bias, int M, int N, int K, int lda,
          int ldb, int ldc, int ta, int tb, int epi) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    if (!p->bf16) {
        k_gemm<TA, TB><<<grid, 256, 0, p->stream>>>(A, B, C, bias, M, N, K, lda, ldb, ldc, ta, tb, epi);
        mck(p, cudaGetLastError(), "gemm");
        return;
    }
    const long long tiles = (long long)grid.x * grid.y;
    int kz = 1;
    if (epi == EPI_NONE && tiles < 152 && K >= 8 * TC_BK) {
        kz = (int)std::min<long long>((8 * 152 + tiles - 1) / tiles, K / (4 * TC_BK));
        kz = (int)std::min<long long>(kz, MLP_SPLITK_WS / ((long long)M * N));
        if (kz < 1) kz = 1;
    }
    int kchunk = (K + kz - 1) / kz;
    kchunk = (kchunk + TC_BK - 1) / TC_BK * TC_BK;
    kz = (K + kchunk - 1) / kchunk;
    grid.z = (unsigned)kz;
    float* out = kz > 1 ? p->ws : C;
    if (std::is_same<TA, __nv_bfloat16>::value && !ta &&
        (lda % 8 != 0 || reinterpret_cast<unsigned long long>(A) % 16 != 0))
        mck(p, cudaErrorInvalidValue, "gemm_tc: BF16 A rows must be 16-byte aligned");
    if (!ta && !tb)
        k_gemm_tc<TA, TB, false, false><<<grid, 128, 0, p->stream>>>(A, B, out, bias, M, N, K, lda, ldb, ldc, epi, kchunk);
    else if (ta && !tb)
        k_gemm_tc<TA, TB, true, false><<<grid, 128, 0, p->stream>>>(A, B, out, bias, M, N, K, lda, ldb, ldc, epi, kchunk);
    else if (!ta && tb)
        k_gemm_tc<TA, TB, false, true><<<grid, 128, 0, p->stream>>>(A, B, out, bias, M, N, K, lda, ldb, ldc, epi, kchunk);
    else
        k_gemm_tc<TA, TB, true, true><<<grid, 128, 0, p->stream>>>(A, B, out, bias, M, N, K, lda, ldb, ldc, epi, kchunk);
    mck(p, cudaGetLastError(), "gemm_tc");
    if (kz > 1) {
        k_splitk_sum<<<ew((long long)M * N), 256, 0, p->stream>>>(p->ws, kz, M, N, C, ldc);
        mck(p, cudaGetLastError(), "splitk_sum");
    }
}

// out[c] = sum over rows of D[row][c] (bias gradients); the split-K
// workspace holds the partial sums
void colsum(sisdc_mlp_s* p, const float* D, int rows, int cols, float* out) {
    const int chunk = (rows + COLSUM_CHUNKS - 1) / COLSUM_CHUNKS;
    const int nchunk = (rows + chunk - 1) / chunk;
    k_colsum_part<<<dim3((cols + 31) / 32, nchunk), dim3(32, 8), 0, p->stream>>>(D, rows, cols, chunk, p->ws);
    k_colsum_fin<<<(cols + 127) / 128, 128, 0, p->stream>>>(p->ws, nchunk, cols, out);
    mck(p, cudaGetLastError(), "colsum");
}

// forward on p->X (rows) -> p->Y; hidden activations kept for backward
void forward(sisdc_mlp_s* p) {
    const int R = (int)p->rows;
    if (p->bf16) {
        gemm<__nv_bfloat16>(p, p->Xb, p->theta_b + p->oW1, p->H1, p->theta + p->ob1, R, p->H, p->n_in, p->ldx, p->H,
                            p->H, 0, 0, EPI_BIAS_TANH);
        gemm<__nv_bfloat16>(p, p->H1, p->theta_b + p->oW2, p->H2, p->theta + p->ob2, R, p->H, p->H, p->H, p->H, p->H,
                            0, 0, EPI_BIAS_TANH);
        gemm<__nv_bfloat16>(p, p->H2, p->theta_b + p->oW3, p->Y, p->theta + p->ob3, R, p->q, p->H, p->H, p->q, p->q,
                            0, 0, EPI_BIAS);
    } else {
        gemm<float>(p, p->X, p->theta + p->oW1, p->H1, p->theta + p->ob1, R, p->H, p->n_in, p->n_in, p->H, p->H, 0, 0,
                    EPI_BIAS_TANH);
        gemm<float>(p, p->H1, p->theta + p->oW2, p->H2, p->theta + p->ob2, R, p->H, p->H, p->H, p->H, p->H, 0, 0,
                    EPI_BIAS_TANH);
        gemm<float>(p, p->H2, p->theta + p->oW3, p->Y, p->theta + p->ob3, R, p->q, p->H, p->H, p->q, p->q, 0, 0,
                    EPI_BIAS);
    }
}

void gather(sisdc_mlp_s* p, const double* field, double c) {
    const float feat = (float)(0.1 * std::log(c / (p->h * p->h)));
    k_mlp_elem_ss<<<ew(p->rows), 256, 0, p->stream>>>(field, p->rows, p->q, p->ss);
    k_mlp_scale<<<ew(p->rows), 256, 0, p->stream>>>(p->ss, p->nex, p->ney, p->q, p->rows, p->s, p->sinv);
    const unsigned fb = (unsigned)std::min<long long>(p->rows, 152LL * 16);
    if (p->bf16)
        k_mlp_fill<__nv_bfloat16><<<fb, FILL_THREADS, 0, p->stream>>>(field, p->sinv, p->nex, p->ney, p->q, p->rows,
                                                                      p->n_in, p->ldx, feat, p->Xb);
    else
        k_mlp_fill<float><<<fb, FILL_THREADS, 0, p->stream>>>(field, p->sinv, p->nex, p->ney, p->q, p->rows, p->n_in,
                                                              p->n_in, feat, p->X);
    mck(p, cudaGetLastError(), "patches");
}

// loss partials (p->part) and gradients (into p->grad) for inputs gathered
// from r and targets dx/s; asynchronous
constexpr int LOSS_NB = 256;
void loss_grad_dev(sisdc_mlp_s* p, const double* r, const double* dx, double c) {
    gather(p, r, c);
    const long long nq = p->rows * p->q;
    k_mlp_targets<<<ew(nq), 256, 0, p->stream>>>(dx, r, p->s, p->q, p->rows, p->T);
    forward(p);
    const int nb = LOSS_NB;
    k_mlp_loss<<<nb, 256, 0, p->stream>>>(p->Y, p->T, nq, 1.f / (float)nq, p->dY, p->part);
    mck(p, cudaGetLastError(), "loss");
    const int R = (int)p->rows;
    float* g = p->grad;
    // layer 3: dW3 = H2^T dY, db3 = colsum dY, dH2 = dY W3^T
    gemm<float>(p, p->H2, p->dY, g + p->oW3, nullptr, p->H, p->q, R, p->H, p->q, p->q, 1, 0, EPI_NONE);
    colsum(p, p->dY, R, p->q, g + p->ob3);
    if (p->bf16)
        gemm<__nv_bfloat16>(p, p->dY, p->theta_b + p->oW3, p->dH, nullptr, R, p->H, p->q, p->q, p->q, p->H, 0, 1,
                            EPI_NONE);
    else
        gemm<float>(p, p->dY, p->theta + p->oW3, p->dH, nullptr, R, p->H, p->q, p->q, p->q, p->H, 0, 1, EPI_NONE);
    k_tanh_back<<<ew((long long)R * p->H), 256, 0, p->stream>>>(p->H2, p->dH, (long long)R * p->H);
    // layer 2
    gemm<float>(p, p->H1, p->dH, g + p->oW2, nullptr, p->H, p->H, R, p->H, p->H, p->H, 1, 0, EPI_NONE);
    colsum(p, p->dH, R, p->H, g + p->ob2);
    // dH1 = dH2 W2^T (reuse H2 as scratch for dH1: H2 no longer needed)
    if (p->bf16)
        gemm<__nv_bfloat16>(p, p->dH, p->theta_b + p->oW2, p->H2, nullptr, R, p->H, p->H, p->H, p->H, p->H, 0, 1,
                            EPI_NONE);
    else
        gemm<float>(p, p->dH, p->theta + p->oW2, p->H2, nullptr, R, p->H, p->H, p->H, p->H, p->H, 0, 1, EPI_NONE);
    k_tanh_back<<<ew((long long)R * p->H), 256, 0, p->stream>>>(p->H1, p->H2, (long long)R * p->H);
    // layer 1
    if (p->bf16)
        gemm<float>(p, p->Xb, p->H2, g + p->oW1, nullptr, p->n_in, p->H, R, p->ldx, p->H, p->H, 1, 0, EPI_NONE);
    else
        gemm<float>(p, p->X, p->H2, g + p->oW1, nullptr, p->n_in, p->H, R, p->n_in, p->H, p->H, 1, 0, EPI_NONE);
    colsum(p, p->H2, R, p->H, g + p->ob1);
    mck(p, cudaGetLastError(), "backward");
}

// loss of one sample set, read back (synchronous)
double loss_grad(sisdc_mlp_s* p, const double* r, const double* dx, double c) {
    loss_grad_dev(p, r, dx, c);
    std::vector<double> hp(LOSS_NB);
    mck(p, cudaMemcpyAsync(hp.data(), p->part, LOSS_NB * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
    mck(p, cudaStreamSynchronize(p->stream), "sync");
    double l = 0.0;
    for (int b = 0; b < LOSS_NB; ++b) l += hp[b];
    return 0.5 * l / (double)(p->rows * p->q);
}

}  // namespace

// Internal accessors of sisdc.cu (level geometry and stream).
namespace sisdc {
void level_shape(sisdc_level lv, int* nc, int* nex, int* ney, int* q, double* hx, double* hy, int* dim);
cudaStream_t level_stream(sisdc_level lv);
}  // namespace sisdc

extern "C" {

sisdc_status sisdc_mlp_create(sisdc_level lv, int hidden, unsigned long long seed, int bf16, sisdc_mlp* out) {
    if (!lv || !out || hidden < 1 || hidden > 4096) return SISDC_E_ARG;
    *out = nullptr;
    sisdc_mlp_s* p = new sisdc_mlp_s();
    int dim = 0;
    double hx = 1, hy = 1;
    level_shape(lv, &p->nc, &p->nex, &p->ney, &p->q, &hx, &hy, &dim);
    if (dim != 2) {
        delete p;
        return SISDC_E_ARG;
    }
    p->lvl = lv;
    p->stream = level_stream(lv);
    p->h = hx < hy ? hx : hy;
    p->H = hidden;
    p->bf16 = bf16 ? 1 : 0;
    p->n_in = 9 * p->q + 1;
    if (p->n_in > FILL_THREADS * FILL_SLOTS) {   // patch gather limit (2D levels have P <= 8)
        delete p;
        return SISDC_E_ARG;
    }
    p->rows = (long long)p->nc * p->nex * p->ney;
    p->oW1 = 0;
    p->ob1 = p->oW1 + (long long)p->n_in * p->H;
    p->oW2 = p->ob1 + p->H;
    p->ob2 = p->oW2 + (long long)p->H * p->H;
    p->oW3 = p->ob2 + p->H;
    p->ob3 = p->oW3 + (long long)p->H * p->q;
    p->nparam = p->ob3 + p->q;
    // deterministic host initialisation (scaled normal via Box-Muller on a
    // splitmix64 stream)
    std::vector<float> w(p->nparam, 0.f);
    unsigned long long st = seed;
    auto nextu = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto normal = [&]() {
        const double u1 = ((nextu() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((nextu() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (long long k = 0; k < (long long)p->n_in * p->H; ++k) w[p->oW1 + k] = (float)(normal() / std::sqrt((double)p->n_in));
    for (long long k = 0; k < (long long)p->H * p->H; ++k) w[p->oW2 + k] = (float)(normal() / std::sqrt((double)p->H));
    for (long long k = 0; k < (long long)p->H * p->q; ++k) w[p->oW3 + k] = (float)(0.1 * normal() / std::sqrt((double)p->H));
    const long long R = p->rows;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    al((void**)&p->theta, p->nparam * sizeof(float));
    al((void**)&p->grad, p->nparam * sizeof(float));
    al((void**)&p->m, p->nparam * sizeof(float));
    al((void**)&p->v, p->nparam * sizeof(float));
    al((void**)&p->theta_b, p->nparam * sizeof(__nv_bfloat16));
    p->ldx = (p->n_in + 7) / 8 * 8;
    if (p->bf16) {
        al((void**)&p->Xb, R * p->ldx * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMemset(p->Xb, 0, R * p->ldx * sizeof(__nv_bfloat16));
    } else {
        al((void**)&p->X, R * p->n_in * sizeof(float));
    }
    al((void**)&p->H1, R * p->H * sizeof(float));
    al((void**)&p->H2, R * p->H * sizeof(float));
    al((void**)&p->dH, R * p->H * sizeof(float));
    al((void**)&p->Y, R * p->q * sizeof(float));
    al((void**)&p->T, R * p->q * sizeof(float));
    al((void**)&p->dY, R * p->q * sizeof(float));
    al((void**)&p->s, R * sizeof(float));
    al((void**)&p->part, 256 * sizeof(double));
    al((void**)&p->ws, MLP_SPLITK_WS * sizeof(float));
    al((void**)&p->ss, R * sizeof(double));
    al((void**)&p->sinv, R * sizeof(float));
    al((void**)&p->lacc, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(p->theta, w.data(), p->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, p->nparam * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(p->v, 0, p->nparam * sizeof(float));
    if (e == cudaSuccess) {
        k_to_bf16<<<ew(p->nparam), 256>>>(p->theta, p->theta_b, p->nparam);
        e = cudaDeviceSynchronize();
    }
    // the tcgen05 forward pass, where the network's shape fits it
    if (e == cudaSuccess && p->bf16 && mlp_tc_eligible(p->n_in, p->H, p->q, nullptr)) {
        p->K1p = (p->n_in + 63) / 64 * 64;
        p->N3 = (p->q + 15) / 16 * 16;
        al((void**)&p->W1T, (size_t)p->H * p->K1p * sizeof(__nv_bfloat16));
        al((void**)&p->W2T, (size_t)p->H * 128 * sizeof(__nv_bfloat16));
        al((void**)&p->W3T, (size_t)p->N3 * 128 * sizeof(__nv_bfloat16));
        al((void**)&p->derr, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->derr, 0, sizeof(int));
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            p->tc_ok = mlp_tc_encode(p->tmap[0], p->W1T, p->H, p->K1p, p->H) &&
                       mlp_tc_encode(p->tmap[1], p->W2T, p->H, 128, p->H) &&
                       mlp_tc_encode(p->tmap[2], p->W3T, p->N3, 128, p->N3);
    }
    if (e != cudaSuccess) {
        sisdc_mlp_destroy(p);
        return e == cudaErrorMemoryAllocation ? SISDC_E_OOM : SISDC_E_CUDA;
    }
    *out = p;
    return SISDC_OK;
}

void sisdc_mlp_destroy(sisdc_mlp p) {
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFree(p->theta); cudaFree(p->grad); cudaFree(p->m); cudaFree(p->v); cudaFree(p->theta_b);
    cudaFree(p->X); cudaFree(p->H1); cudaFree(p->H2); cudaFree(p->dH); cudaFree(p->Y); cudaFree(p->T);
    cudaFree(p->dY); cudaFree(p->s); cudaFree(p->part); cudaFree(p->ws);
    cudaFree(p->ss); cudaFree(p->sinv); cudaFree(p->lacc); cudaFree(p->Xb);
    cudaFree(p->W1T); cudaFree(p->W2T); cudaFree(p->W3T); cudaFree(p->derr);
    delete p;
}

sisdc_status sisdc_mlp_info(sisdc_mlp p, int* n_in, int* hidden, int* n_out, long long* nparam) {
    if (!p) return SISDC_E_ARG;
    if (n_in) *n_in = p->n_in;
    if (hidden) *hidden = p->H;
    if (n_out) *n_out = p->q;
    if (nparam) *nparam = p->nparam;
    return SISDC_OK;
}

sisdc_status sisdc_mlp_params(sisdc_mlp p, float* h_get, const float* h_set) {
    if (!p) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess && h_get) e = cudaMemcpy(h_get, p->theta, p->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_set) {
        e = cudaMemcpy(p->theta, h_set, p->nparam * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            k_to_bf16<<<ew(p->nparam), 256, 0, p->stream>>>(p->theta, p->theta_b, p->nparam);
            e = cudaStreamSynchronize(p->stream);
        }
    }
    return e == cudaSuccess ? SISDC_OK : SISDC_E_CUDA;
}

sisdc_status sisdc_mlp_loss_grad(sisdc_mlp p, const double* d_r, const double* d_dx, double c, double* h_loss,
                                 float* h_grad) {
    if (!p || !d_r || !d_dx || !(c > 0.0)) return SISDC_E_ARG;
    try {
        const double l = loss_grad(p, d_r, d_dx, c);
        if (h_loss) *h_loss = l;
        if (h_grad) mck(p, cudaMemcpy(h_grad, p->grad, p->nparam * sizeof(float), cudaMemcpyDeviceToHost), "copy");
    } catch (const MlpFail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_mlp_train(sisdc_mlp p, const double* d_r, const double* d_dx, const double* h_c, int nsolves,
                             int epochs, double lr, double* h_loss) {
    if (!p || !d_r || !d_dx || !h_c || nsolves < 1 || epochs < 1 || !(lr > 0.0)) return SISDC_E_ARG;
    const long long nv = p->rows * p->q;
    try {
        double last = 0.0;
        for (int ep = 0; ep < epochs; ++ep) {
            // the epoch's losses are summed on the device (fixed order) and read once
            mck(p, cudaMemsetAsync(p->lacc, 0, sizeof(double), p->stream), "memset");
            for (int k = 0; k < nsolves; ++k) {
                if (!(h_c[k] > 0.0)) continue;
                loss_grad_dev(p, d_r + (long long)k * nv, d_dx + (long long)k * nv, h_c[k]);
                k_loss_acc<<<1, 32, 0, p->stream>>>(p->part, LOSS_NB, 0.5 / (double)(p->rows * p->q), p->lacc);
                ++p->adam_t;
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f - std::pow(b1, (float)p->adam_t), c2 = 1.f - std::pow(b2, (float)p->adam_t);
                k_adam<<<ew(p->nparam), 256, 0, p->stream>>>(p->theta, p->grad, p->m, p->v, p->theta_b, p->nparam,
                                                              (float)lr, b1, b2, 1e-8f, c1, c2);
                mck(p, cudaGetLastError(), "adam");
            }
            double sum = 0.0;
            mck(p, cudaMemcpyAsync(&sum, p->lacc, sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
            mck(p, cudaStreamSynchronize(p->stream), "sync");
            last = sum / nsolves;
        }
        mck(p, cudaStreamSynchronize(p->stream), "sync");
        if (h_loss) *h_loss = last;
    } catch (const MlpFail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_mlp_apply(sisdc_mlp p, const double* d_r, double c, double* d_z, int add) {
    if (!p || !d_r || !d_z || !(c > 0.0)) return SISDC_E_ARG;
    try {
        if (p->tc_ok && p->use_tc) {
            // patch scales, then the fused gather + three layers + output on tcgen05
            k_mlp_elem_ss<<<ew(p->rows), 256, 0, p->stream>>>(d_r, p->rows, p->q, p->ss);
            k_mlp_scale<<<ew(p->rows), 256, 0, p->stream>>>(p->ss, p->nex, p->ney, p->q, p->rows, p->s, p->sinv);
            mck(p, mlp_tc_pack(p->theta + p->oW1, p->theta + p->oW2, p->theta + p->oW3, p->n_in, p->H, p->q, p->K1p,
                               p->N3, p->W1T, p->W2T, p->W3T, p->stream), "pack");
            MlpTcArgs a{};
            a.field = d_r; a.sinv = p->sinv; a.s = p->s; a.z = d_z; a.add = add;
            a.b1 = p->theta + p->ob1; a.b2 = p->theta + p->ob2; a.b3 = p->theta + p->ob3;
            a.nex = p->nex; a.ney = p->ney; a.q = p->q; a.n_in = p->n_in; a.H = p->H;
            a.nP1 = p->K1p / 64; a.N3 = p->N3; a.rows = p->rows;
            a.feat = (float)(0.1 * std::log(c / (p->h * p->h)));
            a.err = p->derr;
            mck(p, mlp_tc_forward(a, p->tmap[0], p->tmap[1], p->tmap[2], p->nsm, p->stream), "tcgen05 forward");
            return SISDC_OK;
        }
        gather(p, d_r, c);
        forward(p);
        const long long nq = p->rows * p->q;
        k_mlp_scatter<<<ew(nq), 256, 0, p->stream>>>(p->Y, p->s, d_r, p->q, p->rows, d_z, add);
        mck(p, cudaGetLastError(), "scatter");
    } catch (const MlpFail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_mlp_set_tc(sisdc_mlp p, int enable) {
    if (!p) return SISDC_E_ARG;
    if (enable && !p->tc_ok) {
        p->err = "the tcgen05 forward pass does not fit this network (BF16 mode, hidden width a multiple of 16 "
                 "up to 128, at most 128 outputs) or no TMA encoder";
        return SISDC_E_ARG;
    }
    p->use_tc = enable ? 1 : 0;
    return SISDC_OK;
}

sisdc_status sisdc_mlp_sync(sisdc_mlp p) {
    if (!p) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    int flag = 0;
    if (e == cudaSuccess && p->derr) e = cudaMemcpy(&flag, p->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        p->err = std::string("sync: ") + cudaGetErrorString(e);
        return SISDC_E_CUDA;
    }
    if (flag) {
        cudaMemset(p->derr, 0, sizeof(int));
        p->err = "a wait of the tcgen05 forward pass timed out";
        return SISDC_E_TIMEOUT;
    }
    return SISDC_OK;
}

const char* sisdc_mlp_last_error(sisdc_mlp p) { return p ? p->err.c_str() : "null model"; }

}  // extern "C"
