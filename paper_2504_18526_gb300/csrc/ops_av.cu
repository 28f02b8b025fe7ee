// Persson-Peraire artificial viscosity added to f (Sec. 6: the diffusion
// matrix of the DG right-hand side supplemented by an artificial viscosity;
// Sec. 8: Burgers moving front and Sod shock tube with the parameters d_s,
// c_s).  For n states U_s of a level:
//   k_av_eps   eps_e of every element: modal decay of the sensor component
//              (orthonormal Legendre coefficients of the element's
//              interpolant; energy of the degree-P shell over the total),
//              s = log10 of it, eps = c_s h / P lam_e * ramp(s; s0 =
//              log10(1/P^4), kappa = d_s), lam_e = the element's largest
//              convective spectral radius;
//   k_av_grad  BR1 derivatives of every component: (2/h) D u plus the
//              lifting of the central face value at the element ends;
//   k_av_div   F_s += the same lifted derivative of eps_e * grad u (central
//              face values of eps * g), summed over the directions.
// One block per (state, element) for the sensor (deterministic block sums),
// one thread per (state, component, node) for the two derivative passes.
#include "ops.h"
#include "pde.cuh"

namespace sisdc {

namespace {

__device__ double wave_speed(int pde, const PdeParams& pp, const double* u, int dim) {
    double r = 0.0;
    switch (pde) {
        case 0: r = Pde<0>::rx<double>(pp, u); if (dim == 2) r = fmax(r, Pde<0>::ry<double>(pp, u)); break;
        case 1: r = Pde<1>::rx<double>(pp, u); if (dim == 2) r = fmax(r, Pde<1>::ry<double>(pp, u)); break;
        default: r = Pde<2>::rx<double>(pp, u); if (dim == 2) r = fmax(r, Pde<2>::ry<double>(pp, u)); break;
    }
    return r;
}

__global__ void k_av_eps(const AvArgs a) {
    __shared__ double sq[NQMAX * NQMAX];
    __shared__ double st[NQMAX * NQMAX];
    __shared__ double scratch[32];
    const Geo& g = a.g;
    const int nq = g.nq, q = g.q;
    const long long s = blockIdx.x / g.nel;
    const long long e = blockIdx.x - s * g.nel;
    const double* U = a.U + s * (long long)g.ncomp * g.N;
    const int t = threadIdx.x;
    const bool act = t < q;
    double lam = 0.0;
    if (act) {
        const long long id = e * q + t;
        sq[t] = U[(long long)a.comp * g.N + id];
        double u[4];
        for (int c = 0; c < g.ncomp; ++c) u[c] = U[(long long)c * g.N + id];
        lam = wave_speed(a.pde, PdeParams{a.gamma, a.ax, a.ay}, u, g.dim);
    }
    __syncthreads();
    // x transform of every row: st[j][k] = sum_i Vinv[k][i] q[j][i]
    if (act) {
        const int j = t / nq, k = t - j * nq;
        double v = 0.0;
        for (int i = 0; i < nq; ++i) v += a.vinv[k * nq + i] * sq[j * nq + i];
        st[t] = v;
    }
    __syncthreads();
    double en = 0.0, hi = 0.0;
    if (act) {
        const int l = t / nq, k = t - l * nq;
        double cv = st[t];
        if (g.dim == 2) {                         // y transform: c[l][k] = sum_j Vinv[l][j] st[j][k]
            cv = 0.0;
            for (int j = 0; j < nq; ++j) cv += a.vinv[l * nq + j] * st[j * nq + k];
        }
        en = cv * cv;
        const int P = nq - 1;
        if (k == P || (g.dim == 2 && l == P)) hi = en;
    }
    const double tot = block_sum(en, scratch);
    __syncthreads();
    const double top = block_sum(hi, scratch);
    __syncthreads();
    const double lmax = block_max(lam, scratch);
    if (t == 0) {
        double eps = 0.0;
        if (tot > 0.0 && top > 0.0) {
            const double sv = log10(top / tot);
            double r;
            if (sv < a.s0 - a.kappa) r = 0.0;
            else if (sv > a.s0 + a.kappa) r = 1.0;
            else r = 0.5 * (1.0 + sin(M_PI * (sv - a.s0) / (2.0 * a.kappa)));
            eps = a.eps_scale * lmax * r;
        }
        a.eps[s * g.nel + e] = eps;
    }
}

// lifted derivative of v (per-element factor fe[e] when given) along x (dir
// 0) or y (dir 1) at node (j, i) of element e
__device__ double lifted(const Geo& g, const double* v, const double* fe, long long e, int i, int j, int dir) {
    const int nq = g.nq, q = g.q, P = nq - 1;
    const int ex = (int)(e % g.nex), ey = (int)(e / g.nex);
    const double fo = fe ? fe[e] : 1.0;
    const double* ue = v + e * q;
    double d = 0.0;
    if (dir == 0) {
        for (int k = 0; k < nq; ++k) d += g.D[i * nq + k] * ue[j * nq + k];
        d *= g.sx * fo;
        if (i == P) {
            const long long en = (long long)ey * g.nex + (ex + 1 == g.nex ? 0 : ex + 1);
            const double up = fo * ue[j * nq + P], nb = (fe ? fe[en] : 1.0) * v[en * q + j * nq];
            d += g.liftRx * (0.5 * (up + nb) - up);
        }
        if (i == 0) {
            const long long en = (long long)ey * g.nex + (ex == 0 ? g.nex - 1 : ex - 1);
            const double lo = fo * ue[j * nq], nb = (fe ? fe[en] : 1.0) * v[en * q + j * nq + P];
            d -= g.liftLx * (0.5 * (nb + lo) - lo);
        }
    } else {
        for (int k = 0; k < nq; ++k) d += g.D[j * nq + k] * ue[k * nq + i];
        d *= g.sy * fo;
        if (j == P) {
            const long long en = (long long)(ey + 1 == g.ney ? 0 : ey + 1) * g.nex + ex;
            const double up = fo * ue[P * nq + i], nb = (fe ? fe[en] : 1.0) * v[en * q + i];
            d += g.liftRy * (0.5 * (up + nb) - up);
        }
        if (j == 0) {
            const long long en = (long long)(ey == 0 ? g.ney - 1 : ey - 1) * g.nex + ex;
            const double lo = fo * ue[i], nb = (fe ? fe[en] : 1.0) * v[en * q + P * nq + i];
            d -= g.liftLy * (0.5 * (nb + lo) - lo);
        }
    }
    return d;
}

// grad[s][dir][c][node] = lifted derivative of U_s component c
__global__ void k_av_grad(const AvArgs a) {
    const Geo& g = a.g;
    const long long NV = (long long)g.ncomp * g.N;
    const long long total = (long long)a.n * NV;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx / NV, r = idx - s * NV;
        const long long c = r / g.N, node = r - c * g.N;
        const long long e = node / g.q;
        const int t = (int)(node - e * g.q), j = t / g.nq, i = t - j * g.nq;
        const double* v = a.U + s * NV + c * g.N;
        double* out = a.grad + s * (long long)g.dim * NV;
        out[r] = lifted(g, v, nullptr, e, i, j, 0);
        if (g.dim == 2) out[NV + r] = lifted(g, v, nullptr, e, i, j, 1);
    }
}

// F_s[c][node] += sum over directions of the lifted derivative of eps * g
__global__ void k_av_div(const AvArgs a) {
    const Geo& g = a.g;
    const long long NV = (long long)g.ncomp * g.N;
    const long long total = (long long)a.n * NV;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx / NV, r = idx - s * NV;
        const long long c = r / g.N, node = r - c * g.N;
        const long long e = node / g.q;
        const int t = (int)(node - e * g.q), j = t / g.nq, i = t - j * g.nq;
        const double* eps = a.eps + s * g.nel;
        const double* gr = a.grad + s * (long long)g.dim * NV + c * g.N;
        double d = lifted(g, gr, eps, e, i, j, 0);
        if (g.dim == 2) d += lifted(g, gr + NV, eps, e, i, j, 1);
        a.F[s * NV + r] += d;
    }
}

}  // namespace

cudaError_t launch_av(const AvArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (a.g.q > NQMAX * NQMAX || a.g.ncomp > 4) return cudaErrorInvalidValue;
    const long long blocks_e = (long long)a.n * a.g.nel;
    if (blocks_e > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_av_eps<<<(unsigned)blocks_e, warp_round(a.g.q), 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = (long long)a.n * a.g.ncomp * a.g.N;
    const int block = 256;
    const long long want = (total + block - 1) / block;
    const unsigned grid = (unsigned)(want < 152LL * 32 ? (want > 0 ? want : 1) : 152LL * 32);
    k_av_grad<<<grid, block, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_av_div<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sisdc
