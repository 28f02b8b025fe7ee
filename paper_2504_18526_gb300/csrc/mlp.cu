// Element-patch MLP for the implicit stage: inference, training, learned solve.
//
// Not in the paper (a learned initial guess / preconditioner for the implicit
// equations of Sec. 3.3).  For every element and component the 3x3 element
// patch of a nodal residual field r (9 Q values, neighbour offsets (dy, dx)
// in {-1,0,1}^2 row-major) is scaled by its RMS s and extended by the
// feature 0.1 log(c / h^2); a perceptron n_in -> H -> H -> Q with tanh hidden
// layers predicts the deviation of the centre element's correction from r
// itself (the exact correction as c -> 0): z = r + s MLP(r_patch / s).
// Weights are BF16 (FP32 master copy for training), every product is
// accumulated in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sisdc.h"
#include "ops.h"

namespace sisdc {

// ---- kernels ---------------------------------------------------------------

// one block per row (element-component): gather, RMS scale, feature
__global__ void k_mlp_patches(const double* __restrict__ f, int nc, int nex, int ney, int q, float feat,
                              float* __restrict__ X, float* __restrict__ s, int n_in) {
    __shared__ double scratch[32];
    const long long row = blockIdx.x;
    const int nel = nex * ney;
    const int c = (int)(row / nel);
    const int e = (int)(row - (long long)c * nel);
    const int ex = e % nex, ey = e / nex;
    const long long N = (long long)nel * q;
    double acc = 0.0;
    for (int t = threadIdx.x; t < 9 * q; t += blockDim.x) {
        const int k = t / q, node = t - k * q;
        const int dy = k / 3 - 1, dx = k % 3 - 1;
        const int en = ((ey + dy + ney) % ney) * nex + (ex + dx + nex) % nex;
        const double v = f[c * N + (long long)en * q + node];
        acc += v * v;
    }
    const double tot = block_sum(acc, scratch);
    __shared__ double s_scale;
    if (threadIdx.x == 0) {
        double sc = sqrt(tot / (9.0 * q));
        s_scale = sc > 0.0 ? sc : 1.0;
        s[row] = (float)s_scale;
    }
    __syncthreads();
    const double inv = 1.0 / s_scale;
    float* xr = X + row * n_in;
    for (int t = threadIdx.x; t < 9 * q; t += blockDim.x) {
        const int k = t / q, node = t - k * q;
        const int dy = k / 3 - 1, dx = k % 3 - 1;
        const int en = ((ey + dy + ney) % ney) * nex + (ex + dx + nex) % nex;
        xr[t] = (float)(f[c * N + (long long)en * q + node] * inv);
    }
    if (threadIdx.x == 0) xr[9 * q] = feat;
}

// targets t = (dx - r_centre) / s
__global__ void k_mlp_targets(const double* __restrict__ dx, const double* __restrict__ r, const float* __restrict__ s,
                              int q, long long rows, float* __restrict__ T) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < rows * q; k += (long long)gridDim.x * blockDim.x) {
        const long long row = k / q;
        T[k] = (float)((dx[k] - r[k]) / (double)s[row]);
    }
}

// z (+)= r_centre + s * y (state layout = row-major rows of q values)
__global__ void k_mlp_scatter(const float* __restrict__ Y, const float* __restrict__ s, const double* __restrict__ r,
                              int q, long long rows, double* __restrict__ z, int add) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < rows * q; k += (long long)gridDim.x * blockDim.x) {
        const double v = r[k] + (double)Y[k] * (double)s[k / q];
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

// dH *= (1 - H^2) (tanh derivative)
__global__ void k_tanh_back(const float* __restrict__ H, float* __restrict__ dH, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dH[k] *= 1.f - H[k] * H[k];
}

// column sums (bias gradients), one thread per column, fixed order
__global__ void k_colsum(const float* __restrict__ D, int rows, int cols, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; ++i) s += D[(long long)i * cols + j];
    out[j] = s;
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
    long long adam_t = 0;
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

template <class TB>
void gemm(sisdc_mlp_s* p, const float* A, const TB* B, float* C, const float* bias, int M, int N, int K, int lda,
          int ldb, int ldc, int ta, int tb, int epi) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<float, TB><<<grid, 256, 0, p->stream>>>(A, B, C, bias, M, N, K, lda, ldb, ldc, ta, tb, epi);
    mck(p, cudaGetLastError(), "gemm");
}

// forward on p->X (rows) -> p->Y; hidden activations kept for backward
void forward(sisdc_mlp_s* p) {
    const int R = (int)p->rows;
    if (p->bf16) {
        gemm<__nv_bfloat16>(p, p->X, p->theta_b + p->oW1, p->H1, p->theta + p->ob1, R, p->H, p->n_in, p->n_in, p->H,
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
    k_mlp_patches<<<(unsigned)p->rows, 128, 0, p->stream>>>(field, p->nc, p->nex, p->ney, p->q, feat, p->X, p->s,
                                                            p->n_in);
    mck(p, cudaGetLastError(), "patches");
}

// loss and gradients (into p->grad) for inputs gathered from r and targets dx/s
double loss_grad(sisdc_mlp_s* p, const double* r, const double* dx, double c) {
    gather(p, r, c);
    const long long nq = p->rows * p->q;
    k_mlp_targets<<<ew(nq), 256, 0, p->stream>>>(dx, r, p->s, p->q, p->rows, p->T);
    forward(p);
    const int nb = 256;
    k_mlp_loss<<<nb, 256, 0, p->stream>>>(p->Y, p->T, nq, 1.f / (float)nq, p->dY, p->part);
    mck(p, cudaGetLastError(), "loss");
    const int R = (int)p->rows;
    float* g = p->grad;
    // layer 3: dW3 = H2^T dY, db3 = colsum dY, dH2 = dY W3^T
    gemm<float>(p, p->H2, p->dY, g + p->oW3, nullptr, p->H, p->q, R, p->H, p->q, p->q, 1, 0, EPI_NONE);
    k_colsum<<<(p->q + 127) / 128, 128, 0, p->stream>>>(p->dY, R, p->q, g + p->ob3);
    if (p->bf16)
        gemm<__nv_bfloat16>(p, p->dY, p->theta_b + p->oW3, p->dH, nullptr, R, p->H, p->q, p->q, p->q, p->H, 0, 1,
                            EPI_NONE);
    else
        gemm<float>(p, p->dY, p->theta + p->oW3, p->dH, nullptr, R, p->H, p->q, p->q, p->q, p->H, 0, 1, EPI_NONE);
    k_tanh_back<<<ew((long long)R * p->H), 256, 0, p->stream>>>(p->H2, p->dH, (long long)R * p->H);
    // layer 2
    gemm<float>(p, p->H1, p->dH, g + p->oW2, nullptr, p->H, p->H, R, p->H, p->H, p->H, 1, 0, EPI_NONE);
    k_colsum<<<(p->H + 127) / 128, 128, 0, p->stream>>>(p->dH, R, p->H, g + p->ob2);
    // dH1 = dH2 W2^T (reuse H2 as scratch for dH1: H2 no longer needed)
    if (p->bf16)
        gemm<__nv_bfloat16>(p, p->dH, p->theta_b + p->oW2, p->H2, nullptr, R, p->H, p->H, p->H, p->H, p->H, 0, 1,
                            EPI_NONE);
    else
        gemm<float>(p, p->dH, p->theta + p->oW2, p->H2, nullptr, R, p->H, p->H, p->H, p->H, p->H, 0, 1, EPI_NONE);
    k_tanh_back<<<ew((long long)R * p->H), 256, 0, p->stream>>>(p->H1, p->H2, (long long)R * p->H);
    // layer 1
    gemm<float>(p, p->X, p->H2, g + p->oW1, nullptr, p->n_in, p->H, R, p->n_in, p->H, p->H, 1, 0, EPI_NONE);
    k_colsum<<<(p->H + 127) / 128, 128, 0, p->stream>>>(p->H2, R, p->H, g + p->ob1);
    mck(p, cudaGetLastError(), "backward");
    std::vector<double> hp(nb);
    mck(p, cudaMemcpyAsync(hp.data(), p->part, nb * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
    mck(p, cudaStreamSynchronize(p->stream), "sync");
    double l = 0.0;
    for (int b = 0; b < nb; ++b) l += hp[b];
    return 0.5 * l / (double)nq;
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
    al((void**)&p->X, R * p->n_in * sizeof(float));
    al((void**)&p->H1, R * p->H * sizeof(float));
    al((void**)&p->H2, R * p->H * sizeof(float));
    al((void**)&p->dH, R * p->H * sizeof(float));
    al((void**)&p->Y, R * p->q * sizeof(float));
    al((void**)&p->T, R * p->q * sizeof(float));
    al((void**)&p->dY, R * p->q * sizeof(float));
    al((void**)&p->s, R * sizeof(float));
    al((void**)&p->part, 256 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(p->theta, w.data(), p->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, p->nparam * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(p->v, 0, p->nparam * sizeof(float));
    if (e == cudaSuccess) {
        k_to_bf16<<<ew(p->nparam), 256>>>(p->theta, p->theta_b, p->nparam);
        e = cudaDeviceSynchronize();
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
    cudaFree(p->dY); cudaFree(p->s); cudaFree(p->part);
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
            double sum = 0.0;
            for (int k = 0; k < nsolves; ++k) {
                if (!(h_c[k] > 0.0)) continue;
                sum += loss_grad(p, d_r + (long long)k * nv, d_dx + (long long)k * nv, h_c[k]);
                ++p->adam_t;
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f - std::pow(b1, (float)p->adam_t), c2 = 1.f - std::pow(b2, (float)p->adam_t);
                k_adam<<<ew(p->nparam), 256, 0, p->stream>>>(p->theta, p->grad, p->m, p->v, p->theta_b, p->nparam,
                                                              (float)lr, b1, b2, 1e-8f, c1, c2);
                mck(p, cudaGetLastError(), "adam");
            }
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

const char* sisdc_mlp_last_error(sisdc_mlp p) { return p ? p->err.c_str() : "null model"; }

}  // extern "C"
