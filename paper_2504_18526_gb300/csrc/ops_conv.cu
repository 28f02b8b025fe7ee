// Explicit convective operator c(u) = -div F_c(u) (Sec. 2, Sec. 6), sm_103a.
//
// Strong-form DG-SEM on GLL nodes: the volume part is the sum-factorized
// derivative of the nodal flux, -(2/h_x) D F^x - (2/h_y) F^y D^T, and each
// face node gets the lifting of the Rusanov (local Lax-Friedrichs) flux
//     F* = 1/2 (F(u_L) + F(u_R)) - 1/2 lam (u_R - u_L),
//     lam = max(rho(A_n(u_L)), rho(A_n(u_R))),
// as -(2/h)(1/w_P)(F* - F(u)) on the right face and +(2/h)(1/w_0)(F* - F(u))
// on the left face (and likewise in y).  The same kernel reduces the largest
// convective spectral radius of u (for nu_tilde) and can update the cache of
// c from the previous sweep in place (delta = c_new - c_old).
#include "ops.h"
#include "pde.cuh"

namespace sisdc {

template <int NQ, int DIM, int PDE>
__global__ void k_conv(const ConvArgs a) {
    using P = Pde<PDE>;
    constexpr int NC = P::NC;
    constexpr int NQY = DIM == 2 ? NQ : 1;
    constexpr int Q = NQ * NQY;
    extern __shared__ double sm[];
    double* sD = sm;
    double* sw = sD + NQ * NQ;
    double* scratch = sw + NQ;     // 32
    double* sF = scratch + 32;     // [epb][2][NC][Q]
    const Geo& g = a.g;
    for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) sD[t] = g.D[t];
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) sw[t] = g.w[t];
    const PdeParams pp{a.gamma, a.ax, a.ay};

    const int epb = blockDim.x / Q;
    const int le = threadIdx.x / Q, node = threadIdx.x - le * Q;
    const int i = node % NQ, j = node / NQ;
    const long long e = (long long)blockIdx.x * epb + le;
    const bool act = le < epb && e < g.nel;
    const long long N = g.N;

    double u[NC], Fx[NC], Fy[NC];
    double lmax = 0.0;
    double* sFx = sF + (size_t)le * 2 * NC * Q;
    double* sFy = sFx + NC * Q;
    if (act) {
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = a.u[c * N + e * Q + node];
        P::fx(pp, u, Fx);
        lmax = P::rx(pp, u);
#pragma unroll
        for (int c = 0; c < NC; ++c) sFx[c * Q + node] = Fx[c];
        if (DIM == 2) {
            P::fy(pp, u, Fy);
            lmax = fmax(lmax, P::ry(pp, u));
#pragma unroll
            for (int c = 0; c < NC; ++c) sFy[c * Q + node] = Fy[c];
        }
    }
    __syncthreads();
    if (a.lam) {
        const double bm = block_max(lmax, scratch);
        if (threadIdx.x == 0) atomic_max_nonneg(a.lam, bm);
    }
    if (!act) return;

    double cv[NC];
    const double sx = 2.0 / g.hx;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NQ; ++k) s += sD[i * NQ + k] * sFx[c * Q + j * NQ + k];
        cv[c] = -sx * s;
    }
    if (DIM == 2) {
        const double sy = 2.0 / g.hy;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NQ; ++k) s += sD[j * NQ + k] * sFy[c * Q + k * NQ + i];
            cv[c] -= sy * s;
        }
    }
    const int ei = (int)e, ey = ei / g.nex, ex = ei - ey * g.nex;
    double un[NC], Fs[NC];
    if (i == NQ - 1) {         // right face: own state left, neighbour right
        const long long en = (long long)ey * g.nex + (ex + 1) % g.nex;
#pragma unroll
        for (int c = 0; c < NC; ++c) un[c] = a.u[c * N + en * Q + j * NQ];
        rusanov<PDE, true>(pp, u, un, Fs);
        const double s = sx / sw[NQ - 1];
#pragma unroll
        for (int c = 0; c < NC; ++c) cv[c] -= s * (Fs[c] - Fx[c]);
    }
    if (i == 0) {              // left face: neighbour left, own state right
        const long long en = (long long)ey * g.nex + (ex + g.nex - 1) % g.nex;
#pragma unroll
        for (int c = 0; c < NC; ++c) un[c] = a.u[c * N + en * Q + j * NQ + NQ - 1];
        rusanov<PDE, true>(pp, un, u, Fs);
        const double s = sx / sw[0];
#pragma unroll
        for (int c = 0; c < NC; ++c) cv[c] += s * (Fs[c] - Fx[c]);
    }
    if (DIM == 2) {
        const double sy = 2.0 / g.hy;
        if (j == NQ - 1) {     // top face
            const long long en = (long long)((ey + 1) % g.ney) * g.nex + ex;
#pragma unroll
            for (int c = 0; c < NC; ++c) un[c] = a.u[c * N + en * Q + i];
            rusanov<PDE, false>(pp, u, un, Fs);
            const double s = sy / sw[NQ - 1];
#pragma unroll
            for (int c = 0; c < NC; ++c) cv[c] -= s * (Fs[c] - Fy[c]);
        }
        if (j == 0) {          // bottom face
            const long long en = (long long)((ey + g.ney - 1) % g.ney) * g.nex + ex;
#pragma unroll
            for (int c = 0; c < NC; ++c) un[c] = a.u[c * N + en * Q + (NQ - 1) * NQ + i];
            rusanov<PDE, false>(pp, un, u, Fs);
            const double s = sy / sw[0];
#pragma unroll
            for (int c = 0; c < NC; ++c) cv[c] += s * (Fs[c] - Fy[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const long long idx = c * N + e * Q + node;
        if (a.mode == CONV_DELTA) {
            a.delta[idx] = cv[c] - a.cache[idx];
            a.cache[idx] = cv[c];
        }
        if (a.out) a.out[idx] = cv[c];
    }
}

template <int NQ, int DIM, int PDE>
static cudaError_t conv_impl(const ConvArgs& a, cudaStream_t s) {
    constexpr int NC = Pde<PDE>::NC;
    constexpr int Q = NQ * (DIM == 2 ? NQ : 1);
    const int epb = Q >= 256 ? 1 : 256 / Q;
    const long long grid = (a.g.nel + epb - 1) / epb;
    const size_t sh = (NQ * NQ + NQ + 32 + (size_t)epb * 2 * NC * Q) * sizeof(double);
    k_conv<NQ, DIM, PDE><<<(unsigned)grid, warp_round(epb * Q), sh, s>>>(a);
    return cudaGetLastError();
}

template <int NQ>
static cudaError_t conv_nq(const ConvArgs& a, cudaStream_t s) {
    if (a.g.dim == 1) {
        if (a.pde == 0) return conv_impl<NQ, 1, 0>(a, s);
        return cudaErrorInvalidValue;   // Burgers/Euler here are 2D systems
    }
    switch (a.pde) {
        case 0: return conv_impl<NQ, 2, 0>(a, s);
        case 1: return conv_impl<NQ, 2, 1>(a, s);
        case 2: return conv_impl<NQ, 2, 2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// degrees 9..15: 1D convection-diffusion only
template <int NQ>
static cudaError_t conv_1d(const ConvArgs& a, cudaStream_t s) {
    if (a.g.dim == 1 && a.pde == 0) return conv_impl<NQ, 1, 0>(a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
    switch (a.g.nq) {
        case 10: return conv_1d<10>(a, s);
        case 11: return conv_1d<11>(a, s);
        case 12: return conv_1d<12>(a, s);
        case 13: return conv_1d<13>(a, s);
        case 14: return conv_1d<14>(a, s);
        case 15: return conv_1d<15>(a, s);
        case 16: return conv_1d<16>(a, s);
        case 2: return conv_nq<2>(a, s);
        case 3: return conv_nq<3>(a, s);
        case 4: return conv_nq<4>(a, s);
        case 5: return conv_nq<5>(a, s);
        case 6: return conv_nq<6>(a, s);
        case 7: return conv_nq<7>(a, s);
        case 8: return conv_nq<8>(a, s);
        case 9: return conv_nq<9>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sisdc
