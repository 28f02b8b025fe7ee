// PDE flux definitions shared by the convective-operator kernels (Sec. 2).
#pragma once
#include "common.cuh"

namespace sisdc {

// Parameters the fluxes need (a subset of each kernel's arguments).
struct PdeParams {
    double gamma;
    double ax, ay;
};

template <int PDE>
struct Pde;

template <>
struct Pde<0> {   // scalar convection-diffusion, F = a u
    static constexpr int NC = 1;
    __device__ static void fx(const PdeParams& a, const double* u, double* f) { f[0] = a.ax * u[0]; }
    __device__ static void fy(const PdeParams& a, const double* u, double* f) { f[0] = a.ay * u[0]; }
    __device__ static double rx(const PdeParams& a, const double*) { return fabs(a.ax); }
    __device__ static double ry(const PdeParams& a, const double*) { return fabs(a.ay); }
};

template <>
struct Pde<1> {   // two-component Burgers, F = u (x) u
    static constexpr int NC = 2;
    __device__ static void fx(const PdeParams&, const double* u, double* f) {
        f[0] = u[0] * u[0];
        f[1] = u[0] * u[1];
    }
    __device__ static void fy(const PdeParams&, const double* u, double* f) {
        f[0] = u[0] * u[1];
        f[1] = u[1] * u[1];
    }
    __device__ static double rx(const PdeParams&, const double* u) { return 2.0 * fabs(u[0]); }
    __device__ static double ry(const PdeParams&, const double* u) { return 2.0 * fabs(u[1]); }
};

template <>
struct Pde<2> {   // 2D compressible Euler, perfect gas
    static constexpr int NC = 4;
    __device__ static double pres(const PdeParams& a, const double* u) {
        return (a.gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    }
    __device__ static void fx(const PdeParams& a, const double* u, double* f) {
        const double p = pres(a, u), vx = u[1] / u[0];
        f[0] = u[1];
        f[1] = u[1] * vx + p;
        f[2] = u[2] * vx;
        f[3] = (u[3] + p) * vx;
    }
    __device__ static void fy(const PdeParams& a, const double* u, double* f) {
        const double p = pres(a, u), vy = u[2] / u[0];
        f[0] = u[2];
        f[1] = u[1] * vy;
        f[2] = u[2] * vy + p;
        f[3] = (u[3] + p) * vy;
    }
    __device__ static double rx(const PdeParams& a, const double* u) {
        return fabs(u[1] / u[0]) + sqrt(a.gamma * pres(a, u) / u[0]);
    }
    __device__ static double ry(const PdeParams& a, const double* u) {
        return fabs(u[2] / u[0]) + sqrt(a.gamma * pres(a, u) / u[0]);
    }
};

// Rusanov flux between a left/lower state uL and right/upper state uR.
template <int PDE, bool XDIR>
__device__ __forceinline__ void rusanov(const PdeParams& a, const double* uL, const double* uR,
                                        double* Fs) {
    using P = Pde<PDE>;
    double FL[P::NC], FR[P::NC];
    double lL, lR;
    if (XDIR) {
        P::fx(a, uL, FL);
        P::fx(a, uR, FR);
        lL = P::rx(a, uL);
        lR = P::rx(a, uR);
    } else {
        P::fy(a, uL, FL);
        P::fy(a, uR, FR);
        lL = P::ry(a, uL);
        lR = P::ry(a, uR);
    }
    const double lam = fmax(lL, lR);
#pragma unroll
    for (int c = 0; c < P::NC; ++c) Fs[c] = 0.5 * (FL[c] + FR[c]) - 0.5 * lam * (uR[c] - uL[c]);
}

}  // namespace sisdc
