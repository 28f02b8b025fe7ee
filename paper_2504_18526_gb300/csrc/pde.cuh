// PDE flux definitions shared by the convective-operator kernels (Sec. 2).
// Templated on the arithmetic type T (double for the FP64 path, float for
// the operator evaluations of the mixed-precision path); every constant is
// cast to T so that the float versions stay in FP32.
#pragma once
#include "common.cuh"

namespace sisdc {

// Parameters the fluxes need (a subset of each kernel's arguments), in the
// arithmetic type R of the flux evaluation (converted once per kernel).
template <class R>
struct PdeParamsT {
    R gamma;
    R ax, ay;
};
using PdeParams = PdeParamsT<double>;

template <int PDE>
struct Pde;

template <>
struct Pde<0> {   // scalar convection-diffusion, F = a u
    static constexpr int NC = 1;
    static constexpr bool VISC = false;
    template <class T, class PP> __device__ static void fx(const PP& a, const T* u, T* f) { f[0] = T(a.ax) * u[0]; }
    template <class T, class PP> __device__ static void fy(const PP& a, const T* u, T* f) { f[0] = T(a.ay) * u[0]; }
    template <class T, class PP> __device__ static T rx(const PP& a, const T*) { return fabs(T(a.ax)); }
    template <class T, class PP> __device__ static T ry(const PP& a, const T*) { return fabs(T(a.ay)); }
};

template <>
struct Pde<1> {   // two-component Burgers, F = u (x) u
    static constexpr int NC = 2;
    static constexpr bool VISC = false;
    template <class T, class PP> __device__ static void fx(const PP&, const T* u, T* f) {
        f[0] = u[0] * u[0];
        f[1] = u[0] * u[1];
    }
    template <class T, class PP> __device__ static void fy(const PP&, const T* u, T* f) {
        f[0] = u[0] * u[1];
        f[1] = u[1] * u[1];
    }
    template <class T, class PP> __device__ static T rx(const PP&, const T* u) { return T(2) * fabs(u[0]); }
    template <class T, class PP> __device__ static T ry(const PP&, const T* u) { return T(2) * fabs(u[1]); }
};

template <>
struct Pde<2> {   // 2D compressible Euler, perfect gas
    static constexpr int NC = 4;
    static constexpr bool VISC = false;
    template <class T, class PP> __device__ static T pres(const PP& a, const T* u) {
        return (T(a.gamma) - T(1)) * (u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) / u[0]);
    }
    template <class T, class PP> __device__ static void fx(const PP& a, const T* u, T* f) {
        const T p = pres(a, u), vx = u[1] / u[0];
        f[0] = u[1];
        f[1] = u[1] * vx + p;
        f[2] = u[2] * vx;
        f[3] = (u[3] + p) * vx;
    }
    template <class T, class PP> __device__ static void fy(const PP& a, const T* u, T* f) {
        const T p = pres(a, u), vy = u[2] / u[0];
        f[0] = u[2];
        f[1] = u[1] * vy;
        f[2] = u[2] * vy + p;
        f[3] = (u[3] + p) * vy;
    }
    template <class T, class PP> __device__ static T rx(const PP& a, const T* u) {
        return fabs(u[1] / u[0]) + sqrt(T(a.gamma) * pres(a, u) / u[0]);
    }
    template <class T, class PP> __device__ static T ry(const PP& a, const T* u) {
        return fabs(u[2] / u[0]) + sqrt(T(a.gamma) * pres(a, u) / u[0]);
    }
};

// 2D compressible Navier-Stokes: the Euler fluxes (convective part) plus a
// viscous flux evaluated from the primitive variables w = (v_x, v_y, T),
// T = p / rho, and their gradients (Sec. 2.2; gas constant 1).
template <>
struct Pde<3> : Pde<2> {
    static constexpr bool VISC = true;
    template <class T, class PP> __device__ static void primitive(const PP& a, const T* u, T* w) {
        const T ir = T(1) / u[0];
        w[0] = u[1] * ir;
        w[1] = u[2] * ir;
        w[2] = Pde<2>::pres(a, u) * ir;
    }
    // momentum and energy components of F_v^x (fx) and F_v^y (fy); gx, gy =
    // x and y derivatives of w; tau = mu (grad v + grad v^T - 2/3 div v I)
    template <class T>
    __device__ static void vflux(T mu, T kappa, const T* w, const T* gx, const T* gy, T* fx, T* fy) {
        const T div = gx[0] + gy[1];
        const T txx = mu * (T(2) * gx[0] - (T(2) / T(3)) * div);
        const T tyy = mu * (T(2) * gy[1] - (T(2) / T(3)) * div);
        const T txy = mu * (gy[0] + gx[1]);
        fx[0] = txx;
        fx[1] = txy;
        fx[2] = w[0] * txx + w[1] * txy + kappa * gx[2];
        fy[0] = txy;
        fy[1] = tyy;
        fy[2] = w[0] * txy + w[1] * tyy + kappa * gy[2];
    }
};

// Rusanov flux between a left/lower state uL and right/upper state uR.
template <int PDE, bool XDIR, class T, class PP>
__device__ __forceinline__ void rusanov(const PP& a, const T* uL, const T* uR, T* Fs) {
    using P = Pde<PDE>;
    T FL[P::NC], FR[P::NC];
    T lL, lR;
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
    const T lam = fmax(lL, lR);
#pragma unroll
    for (int c = 0; c < P::NC; ++c) Fs[c] = T(0.5) * (FL[c] + FR[c]) - T(0.5) * lam * (uR[c] - uL[c]);
}

// Rusanov flux minus the normal flux of the own state, Fs - F(uo), at a face
// node shared with the neighbour state un; own_left: the own state is the
// left/lower one.  Same flux as rusanov(), without forming Fs itself.
template <int PDE, bool XDIR, class T, class PP>
__device__ __forceinline__ void rusanov_jump(const PP& a, const T* uo, const T* un, bool own_left, T* d) {
    using P = Pde<PDE>;
    T Fo[P::NC], Fn[P::NC];
    T lo, ln;
    if (XDIR) {
        P::fx(a, uo, Fo);
        P::fx(a, un, Fn);
        lo = P::rx(a, uo);
        ln = P::rx(a, un);
    } else {
        P::fy(a, uo, Fo);
        P::fy(a, un, Fn);
        lo = P::ry(a, uo);
        ln = P::ry(a, un);
    }
    const T hl = T(0.5) * fmax(lo, ln);
#pragma unroll
    for (int c = 0; c < P::NC; ++c) {
        const T du = own_left ? un[c] - uo[c] : uo[c] - un[c];    // uR - uL
        d[c] = T(0.5) * (Fn[c] - Fo[c]) - hl * du;
    }
}

}  // namespace sisdc
