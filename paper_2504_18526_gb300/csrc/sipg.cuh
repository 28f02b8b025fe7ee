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

}  // namespace sisdc
