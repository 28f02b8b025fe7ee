// Elementwise SDC kernels and space-time transfers (sm_103a).
//
// * lincomb: fused right-hand sides of the SI sweeps (Sec. 3.3, Sec. 4.3).
// * quad:    the S.F product Q_m = dt sum_i w^nn_{m,i} F_i for all m at once
//            (Sec. 3.2, eq. cm:incremental), FP64 accumulation.
// * fnn:     F^nn_m(U) = U_m - U_{m-1} - Q_m (eq. cm:incremental:op) and the
//            FAS residual r = g - F^nn(U) (eq. MLSDC:incremental:residual).
// * transfer: I, P, R = I^T as (space (x) space) (x) time tensor products
//            applied per element (Sec. 4.2, Sec. 6.2).
#include "sisdc.h"
#include "ds.cuh"
#include "ops.h"

namespace sisdc {

// one grid barrier that block `absent` skips (failure-detection test)
__global__ void k_barrier_selftest(unsigned* count, unsigned* exits, int* err, int absent,
                                   unsigned long long timeout_ns) {
    if ((int)blockIdx.x != absent) grid_barrier(count, exits, err, timeout_ns);
    grid_exit(count, exits);
}

__global__ void k_convert(int kind, const void* in, long long n, void* out) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        if (kind == 0) {
            static_cast<float*>(out)[t] = d2f_int(static_cast<const double*>(in)[t]);
        } else if (kind == 1) {
            static_cast<double*>(out)[t] = f2d_int(static_cast<const float*>(in)[t]);
        } else if (kind == 2) {
            const dsf v = ds_from_double_int(static_cast<const double*>(in)[t]);
            static_cast<float*>(out)[2 * t] = v.hi;
            static_cast<float*>(out)[2 * t + 1] = v.lo;
        } else {
            const float* p = static_cast<const float*>(in) + 2 * t;
            static_cast<double*>(out)[t] = ds_to_double_int(dsf(p[0], p[1]));
        }
    }
}

static inline unsigned ew_grid(long long n, int bs) {
    long long g = (n + bs - 1) / bs;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__global__ void k_lincomb(const __grid_constant__ LinArgs a) {
    __shared__ double sc[MAXTERMS];
    for (int t = threadIdx.x; t < MAXTERMS; t += blockDim.x) sc[t] = t < a.nterms ? coef_value(a.coef[t]) : 0.0;
    __syncthreads();
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n;
         idx += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int t = 0; t < a.nterms; ++t) v += sc[t] * a.in[t][idx];
        a.out[idx] = v;
    }
}

cudaError_t launch_lincomb(const LinArgs& a, cudaStream_t s) {
    k_lincomb<<<ew_grid(a.n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

struct QuadArgs {
    const void* F;
    int f32;
    double* Q;
    double W[MMAX * MMAX];
    int M;
    double dt;
    long long n;
};

__global__ void k_quad(const __grid_constant__ QuadArgs a) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n;
         idx += (long long)gridDim.x * blockDim.x) {
        double f[MMAX];
        for (int i = 0; i < a.M; ++i)
            f[i] = a.f32 ? (double)static_cast<const float*>(a.F)[i * a.n + idx]
                         : static_cast<const double*>(a.F)[i * a.n + idx];
        for (int m = 0; m < a.M; ++m) {
            double s = 0.0;
            for (int i = 0; i < a.M; ++i) s += a.W[m * a.M + i] * f[i];
            a.Q[m * a.n + idx] = a.dt * s;
        }
    }
}

cudaError_t launch_quad(const void* F, int f32, double* Q, const double* W, int M, double dt, long long n,
                        cudaStream_t s) {
    QuadArgs a;
    a.F = F;
    a.f32 = f32;
    a.Q = Q;
    for (int t = 0; t < M * M; ++t) a.W[t] = W[t];
    a.M = M;
    a.dt = dt;
    a.n = n;
    k_quad<<<ew_grid(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_fnn(const double* u0, const double* U, const double* Q, const double* g, double* r,
                      int M, long long n, int residual) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        double prev = u0[idx];
        for (int m = 0; m < M; ++m) {
            const double cur = U[m * n + idx];
            const double fnn = cur - prev - Q[m * n + idx];
            r[m * n + idx] = residual ? ((g ? g[m * n + idx] : 0.0) - fnn) : fnn;
            prev = cur;
        }
    }
}

cudaError_t launch_fnn(const double* u0, const double* U, const double* Q, const double* g, double* r,
                       int M, long long n, int residual, cudaStream_t s) {
    k_fnn<<<ew_grid(n, 256), 256, 0, s>>>(u0, U, Q, g, r, M, n, residual);
    return cudaGetLastError();
}

__global__ void k_transfer(const TransferArgs a) {
    __shared__ double sS[2 * NQMAX * NQMAX];
    __shared__ double sSy[2 * NQMAX * NQMAX];
    __shared__ double sT[MMAX * MMAX];
    const int rx = a.rx > 1 ? a.rx : 1, ry = a.ry > 1 ? a.ry : 1;
    const bool h = rx > 1 || ry > 1;
    const int nm = a.nqo * a.nqi;
    for (int t = threadIdx.x; t < rx * nm; t += blockDim.x) sS[t] = a.S[t];
    if (h)
        for (int t = threadIdx.x; t < ry * nm; t += blockDim.x) sSy[t] = a.Sy[t];
    for (int t = threadIdx.x; t < a.Mo * a.Mi; t += blockDim.x) sT[t] = a.Tt[t];
    __syncthreads();
    const int qi = a.dim == 2 ? a.nqi * a.nqi : a.nqi;
    const int qo = a.dim == 2 ? a.nqo * a.nqo : a.nqo;
    const long long nel_i = h ? (long long)a.nexi * a.neyi : a.nel;
    const long long nel_o = h ? (long long)a.nexo * a.neyo : a.nel;
    const long long nvi = (long long)a.ncomp * nel_i * qi;
    const long long nvo = (long long)a.ncomp * nel_o * qo;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nvo;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long ec = idx / qo;
        const int node = (int)(idx - ec * qo);
        const int io = node % a.nqo, jo = node / a.nqo;
        double sp[MMAX];
        if (!h) {
            for (int n = 0; n < a.Mi; ++n) {
                const double* in = a.in + n * nvi + ec * qi;
                double s = 0.0;
                if (a.dim == 2) {
                    for (int b = 0; b < a.nqi; ++b) {
                        double t = 0.0;
                        for (int c = 0; c < a.nqi; ++c) t += sS[io * a.nqi + c] * in[b * a.nqi + c];
                        s += sS[jo * a.nqi + b] * t;
                    }
                } else {
                    for (int c = 0; c < a.nqi; ++c) s += sS[io * a.nqi + c] * in[c];
                }
                sp[n] = s;
            }
        } else {
            const long long comp = ec / nel_o;
            const int eo = (int)(ec - comp * nel_o);
            const int exo = eo % a.nexo, eyo = eo / a.nexo;
            // children (input elements) of this output element and their matrices
            const int ncx = a.c2f ? 1 : rx, ncy = a.c2f ? 1 : ry;
            for (int n = 0; n < a.Mi; ++n) {
                double s = 0.0;
                for (int cy = 0; cy < ncy; ++cy)
                    for (int cx = 0; cx < ncx; ++cx) {
                        const int exi = a.c2f ? exo / rx : rx * exo + cx;
                        const int eyi = a.c2f ? eyo / ry : ry * eyo + cy;
                        const int mx = a.c2f ? exo % rx : cx, my = a.c2f ? eyo % ry : cy;
                        const double* in = a.in + n * nvi + (comp * nel_i + (long long)eyi * a.nexi + exi) * qi;
                        const double* Sx = sS + mx * nm;
                        if (a.dim == 2) {
                            const double* Syc = sSy + my * nm;
                            for (int b = 0; b < a.nqi; ++b) {
                                double t = 0.0;
                                for (int c = 0; c < a.nqi; ++c) t += Sx[io * a.nqi + c] * in[b * a.nqi + c];
                                s += Syc[jo * a.nqi + b] * t;
                            }
                        } else {
                            for (int c = 0; c < a.nqi; ++c) s += Sx[io * a.nqi + c] * in[c];
                        }
                    }
                sp[n] = s;
            }
        }
        for (int m = 0; m < a.Mo; ++m) {
            double v = 0.0;
            for (int n = 0; n < a.Mi; ++n) v += sT[m * a.Mi + n] * sp[n];
            double* o = a.out + m * nvo + idx;
            *o = a.add ? *o + v : v;
        }
    }
}

cudaError_t launch_transfer(const TransferArgs& a, cudaStream_t s) {
    const int qo = a.dim == 2 ? a.nqo * a.nqo : a.nqo;
    const bool h = a.rx > 1 || a.ry > 1;
    const long long nel_o = h ? (long long)a.nexo * a.neyo : a.nel;
    k_transfer<<<ew_grid((long long)a.ncomp * nel_o * qo, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---- diagnostics: GLL-weighted L2 norm, discrete mass, max norm -------------
// Deterministic: pass 1 writes one partial per (component, block) in a fixed
// tree order; pass 2 sums the partials of each component in index order.
constexpr int NORM_BLOCKS = 256;

__global__ void k_norms_partial(const Geo g, const double* __restrict__ u, const double* __restrict__ ref,
                                double* part) {
    __shared__ double scratch[32];
    const int c = blockIdx.y;
    const long long n = g.N;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * per, i1 = min(n, i0 + per);
    double s2 = 0.0, s1 = 0.0, mx = 0.0;
    for (long long k = i0 + threadIdx.x; k < i1; k += blockDim.x) {
        const int node = (int)(k % g.q);
        const int i = node % g.nq, j = node / g.nq;
        const double wgt = g.dim == 2 ? (0.5 * g.hx * g.w[i]) * (0.5 * g.hy * g.w[j]) : 0.5 * g.hx * g.w[i];
        const double v = u[c * n + k];
        const double e = ref ? v - ref[c * n + k] : v;
        s2 += wgt * e * e;
        s1 += wgt * v;
        mx = fmax(mx, fabs(e));
    }
    const double t2 = block_sum(s2, scratch);
    const double t1 = block_sum(s1, scratch);
    const double tm = block_max(mx, scratch);
    if (threadIdx.x == 0) {
        double* o = part + ((size_t)c * gridDim.x + blockIdx.x) * 3;
        o[0] = t2;
        o[1] = t1;
        o[2] = tm;
    }
}

__global__ void k_norms_final(const double* part, int nb, double* out) {
    const int c = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s2 = 0.0, s1 = 0.0, mx = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double* o = part + ((size_t)c * nb + b) * 3;
        s2 += o[0];
        s1 += o[1];
        mx = fmax(mx, o[2]);
    }
    out[3 * c + 0] = sqrt(s2);
    out[3 * c + 1] = s1;
    out[3 * c + 2] = mx;
}

int norms_scratch_doubles(int ncomp) { return ncomp * (NORM_BLOCKS * 3 + 3); }

__global__ void k_dot_partial(const Geo g, const double* __restrict__ a, const double* __restrict__ b, int jacobi,
                              double c, double* part) {
    __shared__ double scratch[32];
    const long long n = (long long)g.ncomp * g.N;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * per, i1 = min(n, i0 + per);
    double s = 0.0;
    for (long long k = i0 + threadIdx.x; k < i1; k += blockDim.x) {
        double w = 1.0;
        if (jacobi) {
            const int node = (int)(k % g.q);
            const int i = node % g.nq, j = node / g.nq;
            double mass, dg;
            if (g.dim == 2) {
                const double mx = 0.5 * g.hx * g.w[i], my = 0.5 * g.hy * g.w[j];
                mass = mx * my;
                dg = my * g.dline_x[i] + mx * g.dline_y[j];
            } else {
                mass = 0.5 * g.hx * g.w[i];
                dg = g.dline_x[i];
            }
            w = 1.0 / (mass + c * dg);
        }
        s += a[k] * b[k] * w;
    }
    const double t = block_sum(s, scratch);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_dot_final(const double* part, int nb, double* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    out[0] = s;
}

cudaError_t launch_dot(const Geo& g, const double* a, const double* b, int jacobi, double c, double* scratch,
                       cudaStream_t s) {
    k_dot_partial<<<NORM_BLOCKS, 256, 0, s>>>(g, a, b, jacobi, c, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dot_final<<<1, 32, 0, s>>>(scratch, NORM_BLOCKS, scratch + NORM_BLOCKS);
    return cudaGetLastError();
}

cudaError_t launch_norms(const Geo& g, const double* u, const double* ref, double* scratch, cudaStream_t s) {
    double* part = scratch;
    double* out = scratch + (size_t)g.ncomp * NORM_BLOCKS * 3;
    k_norms_partial<<<dim3(NORM_BLOCKS, g.ncomp), 256, 0, s>>>(g, u, ref, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_norms_final<<<g.ncomp, 32, 0, s>>>(part, NORM_BLOCKS, out);
    return cudaGetLastError();
}

}  // namespace sisdc

extern "C" sisdc_status sisdc_convert(int kind, const void* d_in, long long n, void* d_out, void* cuda_stream) {
    using namespace sisdc;
    if (kind < 0 || kind > 3 || n < 0 || (n > 0 && (!d_in || !d_out))) return SISDC_E_ARG;
    if (n == 0) return SISDC_OK;
    k_convert<<<ew_grid(n, 256), 256, 0, (cudaStream_t)cuda_stream>>>(kind, d_in, n, d_out);
    return cudaGetLastError() == cudaSuccess ? SISDC_OK : SISDC_E_CUDA;
}

extern "C" sisdc_status sisdc_barrier_selftest(int nblocks, int absent, double timeout_ms, void* cuda_stream) {
    using namespace sisdc;
    int dev = 0, nsm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SISDC_E_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop || nblocks < 1 || nblocks > nsm || absent >= nblocks || !(timeout_ms >= 1.0 && timeout_ms <= 2000.0))
        return SISDC_E_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned* words = nullptr;   // count, exits, err
    if (cudaMalloc(&words, 3 * sizeof(unsigned)) != cudaSuccess) return SISDC_E_CUDA;
    sisdc_status out = SISDC_OK;
    if (cudaMemsetAsync(words, 0, 3 * sizeof(unsigned), st) != cudaSuccess) out = SISDC_E_CUDA;
    unsigned* count = words;
    unsigned* exits = words + 1;
    int* err = reinterpret_cast<int*>(words + 2);
    unsigned long long tns = (unsigned long long)(timeout_ms * 1e6);
    void* args[] = {&count, &exits, &err, &absent, &tns};
    if (out == SISDC_OK &&
        cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3((unsigned)nblocks), dim3(32), args, 0, st) !=
            cudaSuccess)
        out = SISDC_E_CUDA;
    int h_err = 0;
    if (out == SISDC_OK && (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                            cudaStreamSynchronize(st) != cudaSuccess))
        out = SISDC_E_CUDA;
    cudaFree(words);
    if (out != SISDC_OK) return out;
    return (h_err & DEV_TIMEOUT) ? SISDC_E_TIMEOUT : SISDC_OK;
}
