// SIPG face lines and operator application for one element (Sec. 6; the
// interior-penalty form of the diffusion operator A, L = -M^-1 A), shared by
// the single-problem and the ensemble sweep kernels.  The geometry type GG
// provides sx, sy (2/h), ihx, ihy (1/h), taux, tauy (penalties) and hx, hy.
#pragma once
#include "common.cuh"

namespace sisdc {

// value and scaled normal derivative at the end of a line of NQ nodes
// normal to face f (f = 0, 1: x faces; 2, 3: y faces)
template <int NQ, class V, class GG>
__device__ __forceinline__ void sipg_face_line(const GG& g, const V* v, int f, const V* Dt, V& val, V& der) {
    const int end = (f & 1) ? NQ - 1 : 0;
    val = v[end];
    V s = V(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) s += Dt[end * NQ + q] * v[q];
    der = s * (f < 2 ? V(g.sx) : V(g.sy));
}

// (A u)(i, j) of one element: u = its Q nodal values, f = its face data
// [face][jump | average][NQ] (jumps [u] and averages {du/dn} of the face
// lines), Dt = D, Kt = D^T W D, wt = GLL weights.
template <int NQ, int DIM, class V, class GG>
__device__ __forceinline__ V sipg_opA(const GG& g, int i, int j, const V* u, const V* f, const V* Dt, const V* Kt,
                                      const V* wt) {
    V ax = V(0);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ax += Kt[i * NQ + k] * u[j * NQ + k];
    ax *= V(g.sx);
    ax -= V(g.ihx) * (Dt[(NQ - 1) * NQ + i] * f[2 * NQ + j] + Dt[i] * f[j]);
    if (i == NQ - 1) ax += -f[3 * NQ + j] + V(g.taux) * f[2 * NQ + j];
    if (i == 0) ax += f[NQ + j] - V(g.taux) * f[j];
    if (DIM == 1) return ax;
    V ay = V(0);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ay += Kt[j * NQ + k] * u[k * NQ + i];
    ay *= V(g.sy);
    ay -= V(g.ihy) * (Dt[(NQ - 1) * NQ + j] * f[6 * NQ + i] + Dt[j] * f[4 * NQ + i]);
    if (j == NQ - 1) ay += -f[7 * NQ + i] + V(g.tauy) * f[6 * NQ + i];
    if (j == 0) ay += f[5 * NQ + i] - V(g.tauy) * f[4 * NQ + i];
    return (V(0.5) * V(g.hy) * wt[j]) * ax + (V(0.5) * V(g.hx) * wt[i]) * ay;
}

// jump [u] and average {du/dn} across face f from the own line vo and the
// neighbour's line vn (both ordered along the normal direction)
template <int NQ, class V, class GG>
__device__ __forceinline__ void sipg_face(const GG& g, const V* vo, const V* vn, int f, const V* Dt, V& jump,
                                          V& avg) {
    V ov, od, nv, nd;
    sipg_face_line<NQ>(g, vo, f, Dt, ov, od);
    sipg_face_line<NQ>(g, vn, f ^ 1, Dt, nv, nd);
    if ((f & 1) == 0) {
        jump = nv - ov;
        avg = V(0.5) * (nd + od);
    } else {
        jump = ov - nv;
        avg = V(0.5) * (od + nd);
    }
}

// Pre-scaled form of sipg_opA for a uniform grid.  The quadrature weights,
// metric factors (2/h, 1/h, h/2) and penalties are folded into one
// coefficient per product, so (A u)(i, j) is a plain sum of products with
// no branches.  cf points at the node's first coefficient and consecutive
// coefficients of a node lie Q apart (layout [coefficient][node]):
//   [0, NQ)            x-direction stiffness row, against u(k, j)
//   [NQ, 2NQ)          y-direction stiffness row, against u(i, k) (2D)
//   DIM*NQ + [0, 4)    x faces: left jump, left average, right jump, right average
//   DIM*NQ + [4, 8)    y faces, same order (2D)
// sipg_opA_coeff gives the coefficient values.
template <int NQ, int DIM, class V>
__device__ __forceinline__ V sipg_opA_pre(int i, int j, const V* u, const V* f, const V* cf) {
    constexpr int Q = DIM == 2 ? NQ * NQ : NQ;
    const V* cx = cf + DIM * NQ * Q;
    V ax = V(0);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ax += cf[k * Q] * u[j * NQ + k];
#pragma unroll
    for (int s = 0; s < 4; ++s) ax += cx[s * Q] * f[s * NQ + j];
    if constexpr (DIM == 1) {
        return ax;
    } else {
        V ay = V(0);
#pragma unroll
        for (int k = 0; k < NQ; ++k) ay += cf[(NQ + k) * Q] * u[k * NQ + i];
#pragma unroll
        for (int s = 0; s < 4; ++s) ay += cx[(4 + s) * Q] * f[(4 + s) * NQ + i];
        return ax + ay;
    }
}

// 2D sipg_opA_pre with coefficients of the unit element (h_x = h_y = 2) and
// the x and y parts returned separately: for an element of sides h_x, h_y,
// (A u)(i, j) = (h_y / h_x) X + (h_x / h_y) Y when the face averages hold
// the unscaled derivatives (face rows D/2, as sipg_face_pre with the unit
// element's half rows gives them).
template <int NQ, class V>
__device__ __forceinline__ void sipg_opA_pre_xy(int i, int j, const V* u, const V* f, const V* cf, V& X, V& Y) {
    constexpr int Q = NQ * NQ;
    const V* cx = cf + 2 * NQ * Q;
    V ax = V(0), ay = V(0);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        ax += cf[k * Q] * u[j * NQ + k];
        ay += cf[(NQ + k) * Q] * u[k * NQ + i];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        ax += cx[s * Q] * f[s * NQ + j];
        ay += cx[(4 + s) * Q] * f[(4 + s) * NQ + i];
    }
    X = ax;
    Y = ay;
}

// geometry of the unit element h_x = h_y = 2 (penalty 2 NQ^2 / h)
struct UnitElementGeo {
    double hx, hy, sx, sy, ihx, ihy, taux, tauy;
    __host__ __device__ constexpr explicit UnitElementGeo(int nq)
        : hx(2.0), hy(2.0), sx(1.0), sy(1.0), ihx(0.5), ihy(0.5), taux(double(nq) * nq), tauy(double(nq) * nq) {}
};

// coefficient k of node (i, j) of sipg_opA_pre (FP64; D, K, w as in sipg_opA)
template <int NQ, int DIM, class GG>
__device__ __forceinline__ double sipg_opA_coeff(const GG& g, const double* D, const double* K, const double* w,
                                                 int k, int i, int j) {
    const double wy = DIM == 2 ? 0.5 * g.hy * w[j] : 1.0;
    const double wx = 0.5 * g.hx * w[i];
    if (k < NQ) return wy * g.sx * K[i * NQ + k];
    if (DIM == 2 && k < 2 * NQ) return wx * g.sy * K[j * NQ + (k - NQ)];
    const int r = k - DIM * NQ;
    const bool xd = r < 4;
    const int a = xd ? i : j, s = r & 3;
    const double wgt = xd ? wy : wx, ih = xd ? g.ihx : g.ihy, tau = xd ? g.taux : g.tauy;
    if (s == 0) return wgt * (-ih * D[a] - (a == 0 ? tau : 0.0));
    if (s == 1) return a == 0 ? wgt : 0.0;
    if (s == 2) return wgt * (-ih * D[(NQ - 1) * NQ + a] + (a == NQ - 1 ? tau : 0.0));
    return a == NQ - 1 ? -wgt : 0.0;
}

// sipg_face with half-scaled end rows: Dh[f][q] = (s/2) D[end(f)][q], s the
// 2/h factor of face f's direction and end(f) the node of face f (0 or NQ-1)
template <int NQ, class V>
__device__ __forceinline__ void sipg_face_pre(const V* vo, const V* vn, int f, const V* Dh, V& jump, V& avg) {
    const V* ro = Dh + f * NQ;
    const V* rn = Dh + (f ^ 1) * NQ;
    V od = V(0), nd = V(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        od += ro[q] * vo[q];
        nd += rn[q] * vn[q];
    }
    const int end = (f & 1) ? NQ - 1 : 0;
    const V ov = vo[end], nv = vn[NQ - 1 - end];
    jump = (f & 1) ? ov - nv : nv - ov;
    avg = od + nd;
}

}  // namespace sisdc
