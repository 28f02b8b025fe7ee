// SIPG diffusion operator and the persistent Jacobi-PCG solve (sm_103a).
//
// The implicit equation of the SI integrators (Sec. 3.3, eq. H_SI(1)),
//     (I - c L) x = rhs   <=>   (M + c A) x = M rhs,   c = dt_m nu_tilde,
// is solved by preconditioned CG in ONE cooperative launch: each block owns a
// fixed set of element tiles for the whole solve, neighbour coupling goes
// through a face-trace buffer (value and normal derivative of every face
// row), and the two inner products per iteration are reduced in a fixed
// order through per-block partials and a bounded grid barrier.
//
// A is the symmetric interior penalty (SIPG) stiffness with GLL quadrature
// on a uniform periodic mesh; on such a mesh it is the Kronecker sum
//     A = (h_y/2 W) (x) A_x + A_y (x) (h_x/2 W)
// of 1D SIPG line operators A_x (volume (2/h) D^T W D, face terms
// -{u'}[v] - {v'}[u] + tau [u][v], tau = 2 (P+1)^2 / h).
#include "ops.h"

namespace sisdc {

template <int NQ, int DIM>
struct Sh {
    static constexpr int NQY = DIM == 2 ? NQ : 1;
    static constexpr int Q = NQ * NQY;
    static constexpr int NF = 2 * DIM;
    static constexpr int TRS = NF * 2 * NQ;   // trace values per element-component
};

template <int NQ>
__device__ __forceinline__ void load_tables(const Geo& g, double* sD, double* sK, double* sw,
                                            double* sdx, double* sdy) {
    for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
        sD[t] = g.D[t];
        sK[t] = g.K[t];
    }
    for (int t = threadIdx.x; t < NQ; t += blockDim.x) {
        sw[t] = g.w[t];
        sdx[t] = g.dline_x[t];
        sdy[t] = g.dline_y[t];
    }
}

// Face traces of a tile held in shared memory: for every face row the value
// and the physical normal-direction derivative (2/h) sum_a D[end][a] u[a].
// Faces: 0 = x-left, 1 = x-right, 2 = y-bottom, 3 = y-top.
template <int NQ, int DIM>
__device__ __forceinline__ void tile_traces(const double* su, int nle, long long ec0, const Geo& g,
                                            const double* sD, double* tr) {
    using S = Sh<NQ, DIM>;
    const int per = S::NF * NQ;
    for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
        const int le = t / per, rem = t - le * per, f = rem / NQ, k = rem - f * NQ;
        if (f < 2 && k >= S::NQY) continue;
        const double* u = su + le * S::Q;
        double val, s = 0.0;
        if (f < 2) {
            const int ie = f == 0 ? 0 : NQ - 1;
            val = u[k * NQ + ie];
#pragma unroll
            for (int a = 0; a < NQ; ++a) s += sD[ie * NQ + a] * u[k * NQ + a];
            s *= 2.0 / g.hx;
        } else {
            const int je = f == 2 ? 0 : NQ - 1;
            val = u[je * NQ + k];
#pragma unroll
            for (int a = 0; a < NQ; ++a) s += sD[je * NQ + a] * u[a * NQ + k];
            s *= 2.0 / g.hy;
        }
        double* o = tr + ((ec0 + le) * S::NF + f) * 2 * NQ;
        o[k] = val;
        o[NQ + k] = s;
    }
}

// Jumps [u] and averages {u'} on the faces of the tile's elements, from the
// trace buffer (neighbours may belong to other blocks: read through L2).
// sf[le][f][0][k] = jump, sf[le][f][1][k] = average.
template <int NQ, int DIM>
__device__ __forceinline__ void tile_faces(const double* tr, long long ec0, int nle, const Geo& g,
                                           double* sf) {
    using S = Sh<NQ, DIM>;
    const int per = S::NF * NQ;
    for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
        const int le = t / per, rem = t - le * per, f = rem / NQ, k = rem - f * NQ;
        if (f < 2 && k >= S::NQY) continue;
        const long long ec = ec0 + le;
        const long long comp = ec / g.nel;
        const int e = (int)(ec - comp * g.nel);
        const int ex = e % g.nex, ey = e / g.nex;
        int en;
        if (f == 0) en = ey * g.nex + (ex + g.nex - 1) % g.nex;
        else if (f == 1) en = ey * g.nex + (ex + 1) % g.nex;
        else if (f == 2) en = ((ey + g.ney - 1) % g.ney) * g.nex + ex;
        else en = ((ey + 1) % g.ney) * g.nex + ex;
        const long long ecn = comp * g.nel + en;
        const int fn = f ^ 1;   // matching face of the neighbour
        const double* own = tr + (ec * S::NF + f) * 2 * NQ;
        const double* nb = tr + (ecn * S::NF + fn) * 2 * NQ;
        const double ov = __ldcg(own + k), od = __ldcg(own + NQ + k);
        const double nv = __ldcg(nb + k), nd = __ldcg(nb + NQ + k);
        double jump, avg;
        if ((f & 1) == 0) {   // neighbour on the left / below
            jump = nv - ov;
            avg = 0.5 * (nd + od);
        } else {              // neighbour on the right / above
            jump = ov - nv;
            avg = 0.5 * (od + nd);
        }
        double* o = sf + ((le * S::NF + f) * 2) * NQ;
        o[k] = jump;
        o[NQ + k] = avg;
    }
}

// (A u) at node (i, j) of one element: sum-factorized volume part plus the
// SIPG face terms of the x and y line operators.
template <int NQ, int DIM>
__device__ __forceinline__ double node_A(const double* u, const double* sf, int i, int j,
                                         const Geo& g, const double* sD, const double* sK,
                                         const double* sw) {
    double ax = 0.0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) ax += sK[i * NQ + k] * u[j * NQ + k];
    ax *= 2.0 / g.hx;
    ax -= (1.0 / g.hx) * (sD[(NQ - 1) * NQ + i] * sf[(1 * 2) * NQ + j] + sD[i] * sf[0 * NQ + j]);
    if (i == NQ - 1) ax += -sf[(1 * 2 + 1) * NQ + j] + g.taux * sf[(1 * 2) * NQ + j];
    if (i == 0) ax += sf[(0 * 2 + 1) * NQ + j] - g.taux * sf[0 * NQ + j];
    if (DIM == 1) return ax;
    double ay = 0.0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) ay += sK[j * NQ + k] * u[k * NQ + i];
    ay *= 2.0 / g.hy;
    ay -= (1.0 / g.hy) * (sD[(NQ - 1) * NQ + j] * sf[(3 * 2) * NQ + i] + sD[j] * sf[(2 * 2) * NQ + i]);
    if (j == NQ - 1) ay += -sf[(3 * 2 + 1) * NQ + i] + g.tauy * sf[(3 * 2) * NQ + i];
    if (j == 0) ay += sf[(2 * 2 + 1) * NQ + i] - g.tauy * sf[(2 * 2) * NQ + i];
    return (0.5 * g.hy * sw[j]) * ax + (0.5 * g.hx * sw[i]) * ay;
}

template <int NQ, int DIM>
__device__ __forceinline__ void node_mass_diag(const Geo& g, const double* sw, const double* sdx,
                                               const double* sdy, int i, int j, double& mass,
                                               double& diagA) {
    if (DIM == 1) {
        mass = 0.5 * g.hx * sw[i];
        diagA = sdx[i];
    } else {
        const double mx = 0.5 * g.hx * sw[i], my = 0.5 * g.hy * sw[j];
        mass = mx * my;
        diagA = my * sdx[i] + mx * sdy[j];
    }
}

// Element-wise fast diagonalisation (the separable preconditioner of the
// implicit SIPG system): z = B_e^{-1} r for every element of the tile, with
// B_e^{-1} = (S_y (x) S_x) diag(f) (S_y (x) S_x)^T, f = 1 / (1 + c (lam_y[j] +
// lam_x[i])) the thread's own factor.  sr holds r on entry (all threads of
// the block call this; both buffers are clobbered); returns z at the
// thread's node.
template <int NQ, int DIM>
__device__ __forceinline__ double tile_fds(double* sr, double* st, const double* sSx, const double* sSy,
                                           double f, int le, int i, int j, bool act) {
    using S = Sh<NQ, DIM>;
    const int base = le * S::Q;
    __syncthreads();
    if (act) {                                    // S_x^T along x
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < NQ; ++a) s += sSx[a * NQ + i] * sr[base + j * NQ + a];
        st[base + j * NQ + i] = DIM == 1 ? s * f : s;
    }
    __syncthreads();
    if (DIM == 2) {
        if (act) {                                // S_y^T along y, scale
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < NQ; ++b) s += sSy[b * NQ + j] * st[base + b * NQ + i];
            sr[base + j * NQ + i] = s * f;
        }
        __syncthreads();
        if (act) {                                // S_y along y
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < NQ; ++b) s += sSy[j * NQ + b] * sr[base + b * NQ + i];
            st[base + j * NQ + i] = s;
        }
        __syncthreads();
    }
    double z = 0.0;
    if (act) {                                    // S_x along x
#pragma unroll
        for (int a = 0; a < NQ; ++a) z += sSx[i * NQ + a] * st[base + j * NQ + a];
    }
    __syncthreads();
    return z;
}

// ---------------------------------------------------------------------------
// Standalone traces / apply kernels
// ---------------------------------------------------------------------------
template <int NQ, int DIM>
__global__ void k_traces(const Geo g, const double* __restrict__ u, double* __restrict__ tr) {
    using S = Sh<NQ, DIM>;
    extern __shared__ double sm[];
    double* sD = sm;
    double* su = sD + NQ * NQ;
    for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) sD[t] = g.D[t];
    const int epb = blockDim.x / S::Q;
    const long long nec = (long long)g.ncomp * g.nel;
    const long long ec0 = (long long)blockIdx.x * epb;
    const int nle = (int)min((long long)epb, nec - ec0);
    const int le = threadIdx.x / S::Q, node = threadIdx.x - le * S::Q;
    if (le < nle) su[le * S::Q + node] = u[(ec0 + le) * S::Q + node];
    __syncthreads();
    tile_traces<NQ, DIM>(su, nle, ec0, g, sD, tr);
}

template <int NQ, int DIM>
__global__ void k_apply(const ApplyArgs a) {
    using S = Sh<NQ, DIM>;
    extern __shared__ double sm[];
    double* sD = sm;
    double* sK = sD + NQ * NQ;
    double* sw = sK + NQ * NQ;
    double* sdx = sw + NQ;
    double* sdy = sdx + NQ;
    double* su = sdy + NQ;
    const int epb = blockDim.x / S::Q;
    double* sf = su + epb * S::Q;
    const Geo& g = a.g;
    load_tables<NQ>(g, sD, sK, sw, sdx, sdy);
    const long long nec = (long long)g.ncomp * g.nel;
    const long long ec0 = (long long)blockIdx.x * epb;
    const int nle = (int)min((long long)epb, nec - ec0);
    const int le = threadIdx.x / S::Q, node = threadIdx.x - le * S::Q;
    const int i = node % NQ, j = node / NQ;
    const bool act = le < nle;
    const long long idx = (ec0 + le) * S::Q + node;
    if (act) su[le * S::Q + node] = a.u[idx];
    tile_faces<NQ, DIM>(a.tr, ec0, nle, g, sf);
    __syncthreads();
    if (!act) return;
    const double Au = node_A<NQ, DIM>(su + le * S::Q, sf + le * S::NF * 2 * NQ, i, j, g, sD, sK, sw);
    double mass, diagA;
    node_mass_diag<NQ, DIM>(g, sw, sdx, sdy, i, j, mass, diagA);
    switch (a.mode) {
        case APPLY_A: a.out[idx] = Au; break;
        case APPLY_LAP: a.out[idx] = -Au / mass; break;
        case APPLY_LAP_F: {
            const double lu = -Au / mass;
            a.out[idx] = lu;
            a.out2[idx] = a.cc[idx] + a.nu * lu;
            break;
        }
        case APPLY_RES:
            a.out[idx] = mass * a.cc[idx] - (mass * su[le * S::Q + node] + coef_value(a.c) * Au);
            break;
        case APPLY_RESN:
            a.out[idx] = a.cc[idx] - (su[le * S::Q + node] + coef_value(a.c) * Au / mass);
            break;
        default: a.out[idx] = mass * su[le * S::Q + node] + coef_value(a.c) * Au; break;
    }
}

// ---------------------------------------------------------------------------
// Persistent cooperative Jacobi-PCG
// ---------------------------------------------------------------------------
template <int NQ, int DIM>
__device__ __forceinline__ void pcg_body(const PCGArgs& a);

template <int NQ, int DIM>
__global__ void __launch_bounds__(1024, 1) k_pcg(const __grid_constant__ PCGArgs a) {
    pcg_body<NQ, DIM>(a);
    grid_exit(a.bar_count, a.bar_exit);
}

template <int NQ, int DIM>
__device__ __forceinline__ void pcg_body(const PCGArgs& a) {
    using S = Sh<NQ, DIM>;
    extern __shared__ double sm[];
    double* sD = sm;
    double* sK = sD + NQ * NQ;
    double* sw = sK + NQ * NQ;
    double* sdx = sw + NQ;
    double* sdy = sdx + NQ;
    double* scratch = sdy + NQ;          // 32
    double* scoef = scratch + 32;        // MAXTERMS
    double* su = scoef + MAXTERMS;
    const int epb = blockDim.x / S::Q;
    double* sf = su + epb * S::Q;
    double* sSx = sf + epb * S::TRS;     // fast-diagonalisation tables and buffer
    double* slx = sSx + NQ * NQ;
    double* sSy = slx + NQ;
    double* sly = sSy + NQ * NQ;
    double* st = sly + NQ;
    const Geo& g = a.g;
    const bool fds = a.prec == PCG_FDS;
    load_tables<NQ>(g, sD, sK, sw, sdx, sdy);
    for (int t = threadIdx.x; t < MAXTERMS; t += blockDim.x) scoef[t] = t < a.nterms ? coef_value(a.coef[t]) : 0.0;
    if (fds)
        for (int t = threadIdx.x; t < 2 * (NQ * NQ + NQ); t += blockDim.x) sSx[t] = g.fds[t];
    __syncthreads();

    const long long nec = (long long)g.ncomp * g.nel;
    const long long ntiles = (nec + epb - 1) / epb;
    const int le = threadIdx.x / S::Q, node = threadIdx.x - le * S::Q;
    const int i = node % NQ, j = node / NQ;
    const int G = gridDim.x;
    const double c = coef_value(a.cimp);
    double mass, diagA;
    node_mass_diag<NQ, DIM>(g, sw, sdx, sdy, i, j, mass, diagA);
    const double dinv = 1.0 / (mass + c * diagA);
    const double ffds = fds ? 1.0 / (1.0 + c * (slx[i] + (DIM == 2 ? sly[j] : 0.0))) : 0.0;
    double* part = a.part;

    // phase 0: r = M b, traces of x, partial b^T D^-1 b
    double acc = 0.0;
    for (long long t = blockIdx.x; t < ntiles; t += G) {
        const long long ec0 = t * epb;
        const int nle = (int)min((long long)epb, nec - ec0);
        const bool act = le < nle;
        const long long idx = (ec0 + le) * S::Q + node;
        double mb = 0.0;
        if (act) {
            double b = 0.0;
            for (int q = 0; q < a.nterms; ++q) b += scoef[q] * a.in[q][idx];
            mb = mass * b;
            a.r[idx] = mb;
            if (!fds) acc += mb * mb * dinv;
            su[le * S::Q + node] = a.x[idx];
        }
        __syncthreads();
        tile_traces<NQ, DIM>(su, nle, ec0, g, sD, a.trx);
        __syncthreads();
        if (fds) {                 // b^T B^-1 b
            if (act) su[le * S::Q + node] = mb;
            const double z = tile_fds<NQ, DIM>(su, st, sSx, sSy, ffds, le, i, j, act);
            if (act) acc += mb * z;
        }
    }
    {
        const double bs = block_sum(acc, scratch);
        if (threadIdx.x == 0) part[blockIdx.x] = bs;
    }
    if (!grid_barrier(a.bar_count, a.bar_exit, a.err)) return;

    // phase 1: r = M b - (M + cA) x, z = D^-1 r, p = z, traces of p
    acc = 0.0;
    for (long long t = blockIdx.x; t < ntiles; t += G) {
        const long long ec0 = t * epb;
        const int nle = (int)min((long long)epb, nec - ec0);
        const bool act = le < nle;
        const long long idx = (ec0 + le) * S::Q + node;
        if (act) su[le * S::Q + node] = a.x[idx];
        tile_faces<NQ, DIM>(a.trx, ec0, nle, g, sf);
        __syncthreads();
        double z = 0.0, rr = 0.0;
        if (act) {
            const double xv = su[le * S::Q + node];
            const double Ax = node_A<NQ, DIM>(su + le * S::Q, sf + le * S::NF * 2 * NQ, i, j, g, sD, sK, sw);
            rr = a.r[idx] - (mass * xv + c * Ax);
            a.r[idx] = rr;
            if (!fds) {
                z = rr * dinv;
                a.p[idx] = z;
                acc += rr * z;
            }
        }
        if (fds) {
            __syncthreads();       // every thread has read x from su
            if (act) su[le * S::Q + node] = rr;
            z = tile_fds<NQ, DIM>(su, st, sSx, sSy, ffds, le, i, j, act);
            if (act) {
                a.p[idx] = z;
                acc += rr * z;
            }
        }
        __syncthreads();
        if (act) su[le * S::Q + node] = z;
        __syncthreads();
        tile_traces<NQ, DIM>(su, nle, ec0, g, sD, a.trp);
        __syncthreads();
    }
    {
        const double bs = block_sum(acc, scratch);
        if (threadIdx.x == 0) part[G + blockIdx.x] = bs;
    }
    if (!grid_barrier(a.bar_count, a.bar_exit, a.err)) return;
    const double bb = grid_total(part, scratch);
    double rz = grid_total(part + G, scratch);
    const double tol2 = fmax(a.rtol * a.rtol * bb, 1e-300);
    int it = 0;
    bool fin = isfinite(rz) && isfinite(bb);

    while (fin && rz > tol2 && it < a.maxit) {
        // phase 2: Ap = (M + cA) p, partial p^T A p
        acc = 0.0;
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long ec0 = t * epb;
            const int nle = (int)min((long long)epb, nec - ec0);
            const bool act = le < nle;
            const long long idx = (ec0 + le) * S::Q + node;
            if (act) su[le * S::Q + node] = a.p[idx];
            tile_faces<NQ, DIM>(a.trp, ec0, nle, g, sf);
            __syncthreads();
            if (act) {
                const double pv = su[le * S::Q + node];
                const double Ap = mass * pv + c * node_A<NQ, DIM>(su + le * S::Q, sf + le * S::NF * 2 * NQ,
                                                                  i, j, g, sD, sK, sw);
                a.Ap[idx] = Ap;
                acc += pv * Ap;
            }
            __syncthreads();
        }
        {
            const double bs = block_sum(acc, scratch);
            if (threadIdx.x == 0) part[2 * G + blockIdx.x] = bs;
        }
        if (!grid_barrier(a.bar_count, a.bar_exit, a.err)) return;
        const double alpha = rz / grid_total(part + 2 * G, scratch);

        // phase 3: x += alpha p, r -= alpha Ap, partial r^T z
        acc = 0.0;
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long ec0 = t * epb;
            const int nle = (int)min((long long)epb, nec - ec0);
            const bool act = le < nle;
            const long long idx = (ec0 + le) * S::Q + node;
            double rr = 0.0;
            if (act) {
                a.x[idx] += alpha * a.p[idx];
                rr = a.r[idx] - alpha * a.Ap[idx];
                a.r[idx] = rr;
                if (!fds) acc += rr * (rr * dinv);
            }
            if (fds) {             // z = B^-1 r, kept for the next search direction
                if (act) su[le * S::Q + node] = rr;
                const double z = tile_fds<NQ, DIM>(su, st, sSx, sSy, ffds, le, i, j, act);
                if (act) {
                    a.z[idx] = z;
                    acc += rr * z;
                }
            }
        }
        {
            const double bs = block_sum(acc, scratch);
            if (threadIdx.x == 0) part[3 * G + blockIdx.x] = bs;
        }
        if (!grid_barrier(a.bar_count, a.bar_exit, a.err)) return;
        const double rzn = grid_total(part + 3 * G, scratch);
        const double beta = rzn / rz;
        rz = rzn;
        ++it;
        fin = isfinite(rz);
        if (!fin || !(rz > tol2) || it >= a.maxit) break;

        // phase 4: p = z + beta p, traces of p
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long ec0 = t * epb;
            const int nle = (int)min((long long)epb, nec - ec0);
            const bool act = le < nle;
            const long long idx = (ec0 + le) * S::Q + node;
            if (act) {
                const double pn = (fds ? a.z[idx] : a.r[idx] * dinv) + beta * a.p[idx];
                a.p[idx] = pn;
                su[le * S::Q + node] = pn;
            }
            __syncthreads();
            tile_traces<NQ, DIM>(su, nle, ec0, g, sD, a.trp);
            __syncthreads();
        }
        if (!grid_barrier(a.bar_count, a.bar_exit, a.err)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.iters_out) *a.iters_out = it;
        atomicAdd((unsigned long long*)&a.stats[ST_SOLVES], 1ull);
        atomicAdd((unsigned long long*)&a.stats[ST_ITERS], (unsigned long long)it);
        atomicMax((unsigned long long*)&a.stats[ST_MAXIT], (unsigned long long)it);
        if (!fin) {
            atomicOr(a.err, DEV_NONFINITE);
        } else if (rz > tol2) {
            atomicOr(a.err, DEV_NOCONV);
            atomicAdd((unsigned long long*)&a.stats[ST_NOCONV], 1ull);
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
#define SISDC_NQ_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9)
// degrees 9..15: 1D levels only
#define SISDC_NQ1D_CASES(X) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

template <int NQ, int DIM>
static cudaError_t traces_impl(const Geo& g, const double* u, double* tr, cudaStream_t s) {
    using S = Sh<NQ, DIM>;
    const int epb = S::Q >= 256 ? 1 : 256 / S::Q;
    const long long nec = (long long)g.ncomp * g.nel;
    const long long grid = (nec + epb - 1) / epb;
    const size_t sh = (NQ * NQ + (size_t)epb * S::Q) * sizeof(double);
    k_traces<NQ, DIM><<<(unsigned)grid, epb * S::Q, sh, s>>>(g, u, tr);
    return cudaGetLastError();
}

cudaError_t launch_traces(const Geo& g, const double* u, double* tr, cudaStream_t s) {
#define X(n) case n: return g.dim == 1 ? traces_impl<n, 1>(g, u, tr, s) : traces_impl<n, 2>(g, u, tr, s);
#define X1(n) case n: return g.dim == 1 ? traces_impl<n, 1>(g, u, tr, s) : cudaErrorInvalidValue;
    switch (g.nq) { SISDC_NQ_CASES(X) SISDC_NQ1D_CASES(X1) default: return cudaErrorInvalidValue; }
#undef X1
#undef X
}

template <int NQ, int DIM>
static cudaError_t apply_impl(const ApplyArgs& a, cudaStream_t s) {
    using S = Sh<NQ, DIM>;
    const int epb = S::Q >= 256 ? 1 : 256 / S::Q;
    const long long nec = (long long)a.g.ncomp * a.g.nel;
    const long long grid = (nec + epb - 1) / epb;
    const size_t sh = (2 * NQ * NQ + 3 * NQ + (size_t)epb * S::Q + (size_t)epb * S::TRS) * sizeof(double);
    k_apply<NQ, DIM><<<(unsigned)grid, epb * S::Q, sh, s>>>(a);
    return cudaGetLastError();
}

// out = M^-1 in (the diagonal GLL mass of every node), for all components
__global__ void k_minv(const Geo g, const double* __restrict__ in, double* __restrict__ out) {
    const long long n = (long long)g.ncomp * g.N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(idx % g.q), j = t / g.nq, i = t - j * g.nq;
        double mass = 0.5 * g.hx * g.w[i];
        if (g.dim == 2) mass *= 0.5 * g.hy * g.w[j];
        out[idx] = in[idx] / mass;
    }
}

cudaError_t launch_minv(const Geo& g, const double* in, double* out, cudaStream_t s) {
    const long long n = (long long)g.ncomp * g.N;
    const long long want = (n + 255) / 256;
    const unsigned grid = (unsigned)(want < 152LL * 32 ? (want > 0 ? want : 1) : 152LL * 32);
    k_minv<<<grid, 256, 0, s>>>(g, in, out);
    return cudaGetLastError();
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s) {
#define X(n) case n: return a.g.dim == 1 ? apply_impl<n, 1>(a, s) : apply_impl<n, 2>(a, s);
#define X1(n) case n: return a.g.dim == 1 ? apply_impl<n, 1>(a, s) : cudaErrorInvalidValue;
    switch (a.g.nq) { SISDC_NQ_CASES(X) SISDC_NQ1D_CASES(X1) default: return cudaErrorInvalidValue; }
#undef X1
#undef X
}

template <int NQ, int DIM>
static size_t pcg_smem(int epb) {
    using S = Sh<NQ, DIM>;
    return (2 * NQ * NQ + 3 * NQ + 32 + MAXTERMS + (size_t)epb * S::Q + (size_t)epb * S::TRS +
            2 * (NQ * NQ + NQ) + (size_t)epb * S::Q) * sizeof(double);
}

template <int NQ, int DIM>
static int pcg_grid_impl(const Geo& g, int* block) {
    using S = Sh<NQ, DIM>;
    const int epb = S::Q >= 1024 ? 1 : 1024 / S::Q;
    const int bs = warp_round(epb * S::Q);   // in-kernel epb = blockDim / Q is unchanged (epb is maximal)
    const size_t sh = pcg_smem<NQ, DIM>(epb);
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (sh > 48 * 1024)
        cudaFuncSetAttribute(k_pcg<NQ, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg<NQ, DIM>, bs, sh) != cudaSuccess || per < 1)
        return 0;
    const long long nec = (long long)g.ncomp * g.nel;
    const long long ntiles = (nec + epb - 1) / epb;
    long long grid = (long long)per * nsm;
    if (grid > ntiles) grid = ntiles;
    *block = bs;
    return (int)grid;
}

int pcg_grid(const Geo& g, int* block) {
#define X(n) case n: return g.dim == 1 ? pcg_grid_impl<n, 1>(g, block) : pcg_grid_impl<n, 2>(g, block);
#define X1(n) case n: return g.dim == 1 ? pcg_grid_impl<n, 1>(g, block) : 0;
    switch (g.nq) { SISDC_NQ_CASES(X) SISDC_NQ1D_CASES(X1) default: return 0; }
#undef X1
#undef X
}

template <int NQ, int DIM>
static cudaError_t pcg_impl(const PCGArgs& a, int grid, int block, cudaStream_t s) {
    using S = Sh<NQ, DIM>;
    const int epb = block / S::Q;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = pcg_smem<NQ, DIM>(epb);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg<NQ, DIM>, a);
}

cudaError_t launch_pcg(const PCGArgs& a, int grid, int block, cudaStream_t s) {
#define X(n) case n: return a.g.dim == 1 ? pcg_impl<n, 1>(a, grid, block, s) : pcg_impl<n, 2>(a, grid, block, s);
#define X1(n) case n: return a.g.dim == 1 ? pcg_impl<n, 1>(a, grid, block, s) : cudaErrorInvalidValue;
    switch (a.g.nq) { SISDC_NQ_CASES(X) SISDC_NQ1D_CASES(X1) default: return cudaErrorInvalidValue; }
#undef X1
#undef X
}

}  // namespace sisdc
