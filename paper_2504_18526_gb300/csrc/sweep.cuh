// Persistent cooperative SI-SDC sweep kernel (sm_103a).
//
// One launch runs a whole predictor sweep (eqs. sdc:incremental_predictor_si1
// and _si2), `nsweeps` incremental correction sweeps (Algorithm 1 with the
// SI(1)/SI(2) deltas, Sec. 3.3 and Sec. 4.3), or the cache refresh that makes
// f(U), c(U) and L U consistent with a new iterate.  Every block owns a fixed
// set of elements (all components) for the whole launch, so elementwise work
// (right-hand sides, the S.F quadrature, CG vector updates, f updates) needs
// no synchronisation; only neighbour coupling (face values of c(u), SIPG face
// traces) and global reductions (CG inner products, the largest spectral
// radius entering nu_tilde) go through the bounded grid barrier.  Data other
// blocks write during the launch is read through L2 (__ldcg).
//
// Implicit solves: Jacobi-PCG on (M + c A) x = M b with two barriers per
// iteration.  A block forms the face lines of a neighbour's new search
// direction p_new = D^-1 r + beta p_old itself, from the neighbour's r and
// p_old (p is double-buffered), with the same inline arithmetic the owner
// uses, so both sides of every face see bitwise-identical values and p never
// has to be published before it is used.
#pragma once
#include "ops.h"
#include "pde.cuh"

namespace sisdc {

template <int NQ, int DIM, int PDE>
struct Sweeper {
    using PD = Pde<PDE>;
    static constexpr int NC = PD::NC;
    static constexpr int NQY = DIM == 2 ? NQ : 1;
    static constexpr int Q = NQ * NQY;
    static constexpr int NF = 2 * DIM;
    static constexpr int TRS = NF * 2 * NQ;

    const SweepArgs& a;
    const Geo& g;
    PdeParams pp;
    double *sD, *sK, *sw, *sdx, *sdy, *scratch, *su, *sf, *sF, *slam_old, *slam_new, *sdinv;
    int epb, le, node, i, j, G;
    long long ntiles, N;
    double mass, diagA;
    int solve_parity;

    struct Terms {
        int n;
        const double* in[6];
        double cf[6];
        __device__ void add(const double* p, double c) {
            in[n] = p;
            cf[n] = c;
            ++n;
        }
    };

    __device__ Sweeper(const SweepArgs& args) : a(args), g(args.g) {
        extern __shared__ double sm[];
        pp = PdeParams{a.gamma, a.ax, a.ay};
        epb = a.epb;
        sD = sm;
        sK = sD + NQ * NQ;
        sw = sK + NQ * NQ;
        sdx = sw + NQ;
        sdy = sdx + NQ;
        scratch = sdy + NQ;
        slam_old = scratch + 32;
        slam_new = slam_old + MMAX + 1;
        sdinv = slam_new + MMAX + 1;          // [Q] Jacobi factors of the current solve
        su = sdinv + Q;                       // [epb][NC][Q]
        sf = su + epb * NC * Q;               // [epb][NC][NF][2][NQ]
        sF = sf + epb * NC * TRS;             // [epb][2][NC][Q]
        for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
            sD[t] = g.D[t];
            sK[t] = g.K[t];
        }
        for (int t = threadIdx.x; t < NQ; t += blockDim.x) {
            sw[t] = g.w[t];
            sdx[t] = g.dline_x[t];
            sdy[t] = g.dline_y[t];
        }
        for (int t = threadIdx.x; t <= MMAX; t += blockDim.x) {
            slam_old[t] = __ldcg(a.lam + t);
            slam_new[t] = __ldcg(a.lam + MMAX + 1 + t);
        }
        le = threadIdx.x / Q;
        node = threadIdx.x - le * Q;
        i = node % NQ;
        j = node / NQ;
        G = gridDim.x;
        ntiles = (g.nel + epb - 1) / epb;
        N = g.N;
        solve_parity = 0;
        __syncthreads();
        mass_diag(i, j, mass, diagA);
    }

    // GLL mass and diagonal of A at node (ii, jj) of an element
    __device__ void mass_diag(int ii, int jj, double& ms, double& dg) const {
        if (DIM == 1) {
            ms = 0.5 * g.hx * sw[ii];
            dg = sdx[ii];
        } else {
            const double mx = 0.5 * g.hx * sw[ii], my = 0.5 * g.hy * sw[jj];
            ms = mx * my;
            dg = my * sdx[ii] + mx * sdy[jj];
        }
    }

    __device__ bool bar() { return grid_barrier(a.bar_count, a.bar_gen, a.err); }

    __device__ void put_partial(double* slot, double v) {
        const double s = block_sum(v, scratch);
        if (threadIdx.x == 0) slot[blockIdx.x] = s;
    }
    __device__ void put_partial_max(double* slot, double v) {
        const double s = block_max(v, scratch);
        if (threadIdx.x == 0) slot[blockIdx.x] = s;
    }
    __device__ double total(const double* slot) { return grid_total(slot, scratch); }
    __device__ double total_max(const double* slot) {
        __shared__ double s_tot;
        if (threadIdx.x < 32) {
            double v = 0.0;
            for (int b = threadIdx.x; b < G; b += 32) v = fmax(v, __ldcg(slot + b));
            v = warp_max(v);
            if (threadIdx.x == 0) s_tot = v;
        }
        __syncthreads();
        const double r = s_tot;
        __syncthreads();
        return r;
    }

    // ---- tile helpers -------------------------------------------------------
    __device__ long long vidx(int c, long long e) const { return c * N + e * Q + node; }

    __device__ long long neighbour(long long e, int f) const {
        const int ex = (int)(e % g.nex), ey = (int)(e / g.nex);
        if (f == 0) return (long long)ey * g.nex + (ex + g.nex - 1) % g.nex;
        if (f == 1) return (long long)ey * g.nex + (ex + 1) % g.nex;
        if (f == 2) return (long long)((ey + g.ney - 1) % g.ney) * g.nex + ex;
        return (long long)((ey + 1) % g.ney) * g.nex + ex;
    }

    // node of the line normal to face f through face row k, position q
    __device__ static int line_node(int f, int k, int q) { return f < 2 ? k * NQ + q : q * NQ + k; }

    // value and physical normal derivative at the face end of a line
    __device__ void face_line(const double* v, int f, double& val, double& der) const {
        const int end = (f & 1) ? NQ - 1 : 0;
        val = v[end];
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += sD[end * NQ + q] * v[q];
        der = s * (f < 2 ? g.sx : g.sy);
    }

    // jumps [u] and averages {u'} on the faces of the tile's elements: own
    // lines from the tile in su, neighbour lines from getv(c, e, node).
    template <class GetV>
    __device__ void faces(int nle, long long e0, GetV getv) {
        const int per = NC * NF * NQ;
        for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
            const int l = t / per;
            int rem = t - l * per;
            const int c = rem / (NF * NQ);
            rem -= c * NF * NQ;
            const int f = rem / NQ, k = rem - f * NQ;
            if (f < 2 && k >= NQY) continue;
            const long long en = neighbour(e0 + l, f);
            const double* u = su + (l * NC + c) * Q;
            double vo[NQ], vn[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                vo[q] = u[line_node(f, k, q)];
                vn[q] = getv(c, en, line_node(f ^ 1, k, q));
            }
            double ov, od, nv, nd;
            face_line(vo, f, ov, od);
            face_line(vn, f ^ 1, nv, nd);
            double jump, avg;
            if ((f & 1) == 0) {
                jump = nv - ov;
                avg = 0.5 * (nd + od);
            } else {
                jump = ov - nv;
                avg = 0.5 * (od + nd);
            }
            double* o = sf + ((l * NC + c) * NF + f) * 2 * NQ;
            o[k] = jump;
            o[NQ + k] = avg;
        }
    }

    // new search direction at one node (shared by owner and neighbours)
    __device__ static double pnew(double r, double dinv, double beta, double pold) {
        const double z = r * dinv;
        return beta == 0.0 ? z : z + beta * pold;
    }

    // (A u)(i, j) for component c of local element l (tile in su, faces in sf)
    __device__ double opA(int l, int c) const {
        const double* u = su + (l * NC + c) * Q;
        const double* f = sf + (l * NC + c) * TRS;
        double ax = 0.0;
#pragma unroll
        for (int k = 0; k < NQ; ++k) ax += sK[i * NQ + k] * u[j * NQ + k];
        ax *= g.sx;
        ax -= g.ihx * (sD[(NQ - 1) * NQ + i] * f[2 * NQ + j] + sD[i] * f[j]);
        if (i == NQ - 1) ax += -f[3 * NQ + j] + g.taux * f[2 * NQ + j];
        if (i == 0) ax += f[NQ + j] - g.taux * f[j];
        if (DIM == 1) return ax;
        double ay = 0.0;
#pragma unroll
        for (int k = 0; k < NQ; ++k) ay += sK[j * NQ + k] * u[k * NQ + i];
        ay *= g.sy;
        ay -= g.ihy * (sD[(NQ - 1) * NQ + j] * f[6 * NQ + i] + sD[j] * f[4 * NQ + i]);
        if (j == NQ - 1) ay += -f[7 * NQ + i] + g.tauy * f[6 * NQ + i];
        if (j == 0) ay += f[5 * NQ + i] - g.tauy * f[4 * NQ + i];
        return (0.5 * g.hy * sw[j]) * ax + (0.5 * g.hx * sw[i]) * ay;
    }

    // run f(e0, nle) over the block's element tiles
    template <class F>
    __device__ void tiles(F f) {
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long e0 = t * epb;
            f(e0, (int)min((long long)epb, (long long)g.nel - e0));
        }
    }

    // ---- implicit solve -------------------------------------------------------
    // (M + c A) x = M b, b = sum_t cf_t in_t.  The initial guess is xsrc (x
    // itself when xsrc == x); neighbours' xsrc must be final on entry.
    __device__ bool solve(double* x, const double* xsrc, const Terms& tm, double c) {
        double* part = a.part + (size_t)(solve_parity ? 4 : 0) * G;
        solve_parity ^= 1;
        __syncthreads();
        for (int t = threadIdx.x; t < Q; t += blockDim.x) {
            const int ii = t % NQ, jj = t / NQ;
            double ms, dg;
            mass_diag(ii, jj, ms, dg);
            sdinv[t] = 1.0 / (ms + c * dg);
        }
        __syncthreads();
        const double dinv = sdinv[node];
        double acc_bb = 0.0, acc = 0.0;
        tiles([&](const long long e0, const int nle) {
            const bool act = le < nle;
            const long long e = e0 + le;
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    const double xv = __ldcg(xsrc + id);
                    su[(le * NC + cc) * Q + node] = xv;
                    if (xsrc != x) x[id] = xv;
                }
            }
            __syncthreads();
            faces(nle, e0, [&](int cc, long long en, int nd) { return __ldcg(xsrc + cc * N + en * Q + nd); });
            __syncthreads();
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    double b = 0.0;
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        if (q < tm.n) b += tm.cf[q] * __ldcg(tm.in[q] + id);
                    const double mb = mass * b;
                    const double xv = su[(le * NC + cc) * Q + node];
                    const double rr = mb - (mass * xv + c * opA(le, cc));
                    a.r[id] = rr;
                    acc_bb += mb * mb * dinv;
                    acc += rr * (rr * dinv);
                }
            }
            __syncthreads();
        });
        put_partial(part, acc_bb);
        put_partial(part + G, acc);
        if (!bar()) return false;
        const double bb = total(part);
        double rz = total(part + G);
        const double tol2 = fmax(a.rtol * a.rtol * bb, 1e-300);
        bool fin = isfinite(rz) && isfinite(bb);
        int it = 0, par = 0;
        double beta = 0.0;
        while (fin && rz > tol2 && it < a.maxit) {
            const double* pold = par ? a.p2 : a.p;
            double* pcur = par ? a.p : a.p2;
            acc = 0.0;
            tiles([&](const long long e0, const int nle) {
                const bool act = le < nle;
                const long long e = e0 + le;
                double pn[NC];
                if (act) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e);
                        pn[cc] = pnew(__ldcg(a.r + id), dinv, beta, beta == 0.0 ? 0.0 : __ldcg(pold + id));
                        pcur[id] = pn[cc];
                        su[(le * NC + cc) * Q + node] = pn[cc];
                    }
                }
                __syncthreads();
                faces(nle, e0, [&](int cc, long long en, int nd) {
                    const long long id = cc * N + en * Q + nd;
                    return pnew(__ldcg(a.r + id), sdinv[nd], beta, beta == 0.0 ? 0.0 : __ldcg(pold + id));
                });
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const double Apv = mass * pn[cc] + c * opA(le, cc);
                        a.Ap[vidx(cc, e)] = Apv;
                        acc += pn[cc] * Apv;
                    }
                }
                __syncthreads();
            });
            put_partial(part + 2 * G, acc);
            if (!bar()) return false;
            const double alpha = rz / total(part + 2 * G);
            acc = 0.0;
            tiles([&](const long long e0, const int nle) {
                if (le < nle) {
                    const long long e = e0 + le;
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e);
                        x[id] = __ldcg(x + id) + alpha * __ldcg(pcur + id);
                        const double rr = __ldcg(a.r + id) - alpha * __ldcg(a.Ap + id);
                        a.r[id] = rr;
                        acc += rr * (rr * dinv);
                    }
                }
            });
            put_partial(part + 3 * G, acc);
            if (!bar()) return false;
            const double rzn = total(part + 3 * G);
            beta = rzn / rz;
            rz = rzn;
            ++it;
            par ^= 1;
            fin = isfinite(rz);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
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
        return true;
    }

    // ---- convective operator phase -------------------------------------------
    // c(X) for the block's elements; out by mode; optional spectral-radius
    // partial into lamslot; optional traces of X into trout.
    __device__ void conv(const double* X, int mode, double* out, double* lamslot) {
        double lmax = 0.0;
        tiles([&](const long long e0, const int nle) {
            const bool act = le < nle;
            const long long e = e0 + le;
            double u[NC], Fx[NC], Fy[NC];
            double* sFx = sF + (size_t)le * 2 * NC * Q;
            double* sFy = sFx + NC * Q;
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    u[cc] = __ldcg(X + vidx(cc, e));
                    su[(le * NC + cc) * Q + node] = u[cc];
                }
                PD::fx(pp, u, Fx);
                lmax = fmax(lmax, PD::rx(pp, u));
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) sFx[cc * Q + node] = Fx[cc];
                if (DIM == 2) {
                    PD::fy(pp, u, Fy);
                    lmax = fmax(lmax, PD::ry(pp, u));
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) sFy[cc * Q + node] = Fy[cc];
                }
            }
            __syncthreads();
            if (act) {
                double cv[NC];
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < NQ; ++k) s += sD[i * NQ + k] * sFx[cc * Q + j * NQ + k];
                    cv[cc] = -g.sx * s;
                }
                if (DIM == 2) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        double s = 0.0;
#pragma unroll
                        for (int k = 0; k < NQ; ++k) s += sD[j * NQ + k] * sFy[cc * Q + k * NQ + i];
                        cv[cc] -= g.sy * s;
                    }
                }
                double un[NC], Fs[NC];
                if (i == NQ - 1) {
                    const long long en = neighbour(e, 1);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) un[cc] = __ldcg(X + cc * N + en * Q + j * NQ);
                    rusanov<PDE, true>(pp, u, un, Fs);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) cv[cc] -= g.liftRx * (Fs[cc] - Fx[cc]);
                }
                if (i == 0) {
                    const long long en = neighbour(e, 0);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) un[cc] = __ldcg(X + cc * N + en * Q + j * NQ + NQ - 1);
                    rusanov<PDE, true>(pp, un, u, Fs);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) cv[cc] += g.liftLx * (Fs[cc] - Fx[cc]);
                }
                if (DIM == 2) {
                    if (j == NQ - 1) {
                        const long long en = neighbour(e, 3);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) un[cc] = __ldcg(X + cc * N + en * Q + i);
                        rusanov<PDE, false>(pp, u, un, Fs);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) cv[cc] -= g.liftRy * (Fs[cc] - Fy[cc]);
                    }
                    if (j == 0) {
                        const long long en = neighbour(e, 2);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) un[cc] = __ldcg(X + cc * N + en * Q + (NQ - 1) * NQ + i);
                        rusanov<PDE, false>(pp, un, u, Fs);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) cv[cc] += g.liftLy * (Fs[cc] - Fy[cc]);
                    }
                }
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    if (mode == CONV_DELTA) {
                        a.dC[id] = cv[cc] - __ldcg(out + id);
                    }
                    out[id] = cv[cc];
                }
            }
            __syncthreads();
        });
        if (lamslot) put_partial_max(lamslot, lmax);
    }

    // LU = L X, F = CC + nu LU (neighbours' X must be final)
    __device__ void lap(const double* X, double* LUm, double* Fm, const double* CCm) {
        tiles([&](const long long e0, const int nle) {
            const bool act = le < nle;
            const long long e = e0 + le;
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) su[(le * NC + cc) * Q + node] = __ldcg(X + vidx(cc, e));
            }
            __syncthreads();
            faces(nle, e0, [&](int cc, long long en, int nd) { return __ldcg(X + cc * N + en * Q + nd); });
            __syncthreads();
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    const double lu = -opA(le, cc) / mass;
                    LUm[id] = lu;
                    Fm[id] = __ldcg(CCm + id) + a.nu * lu;
                }
            }
            __syncthreads();
        });
    }

    // elementwise: out = sum_t cf_t in_t over the block's nodes
    __device__ void lin(double* out, const Terms& tm) {
        tiles([&](const long long e0, const int nle) {
            if (le < nle) {
                const long long e = e0 + le;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    double v = 0.0;
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        if (q < tm.n) v += tm.cf[q] * __ldcg(tm.in[q] + id);
                    out[id] = v;
                }
            }
        });
    }

    // elementwise S.F quadrature Q_m = dt sum_i W[m][i] F_i (FP64 accumulation)
    __device__ void quad() {
        tiles([&](const long long e0, const int nle) {
            if (le < nle) {
                const long long e = e0 + le;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    double f[MMAX];
#pragma unroll
                    for (int q = 0; q < MMAX; ++q) f[q] = q < a.M ? __ldcg(a.F + q * (NC * N) + id) : 0.0;
#pragma unroll
                    for (int m = 0; m < MMAX; ++m) {
                        if (m >= a.M) break;
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < MMAX; ++q)
                            if (q < a.M) s += a.W[m * a.M + q] * f[q];
                        a.Qb[m * (NC * N) + id] = a.dt * s;
                    }
                }
            }
        });
    }

    __device__ double nut(double dtm, double lam) const { return a.nu_d + 0.5 * dtm * lam * lam; }
    __device__ double* Um(double* U, int m) const { return U + (long long)m * NC * N; }
    __device__ const double* Um(const double* U, int m) const { return U + (long long)m * NC * N; }

    // ---- the three modes ------------------------------------------------------
    __device__ bool refresh() {
        conv(a.u0, CONV_OUT, a.c0, a.partmax);
        for (int m = 0; m < a.M; ++m) {
            conv(Um(a.U, m), CONV_OUT, Um(a.CC, m), a.partmax + (size_t)(m + 1) * G);
            lap(Um(a.U, m), Um(a.LU, m), Um(a.F, m), Um(a.CC, m));
        }
        if (!bar()) return false;
        for (int m = 0; m <= a.M; ++m) {
            const double v = total_max(a.partmax + (size_t)m * G);
            if (threadIdx.x == 0) slam_old[m] = v;
        }
        if (threadIdx.x == 0) slam_new[0] = slam_old[0];
        __syncthreads();
        return true;
    }

    __device__ bool predict() {
        conv(a.u0, CONV_OUT, a.c0, a.partmax);
        if (!bar()) return false;
        double lam = total_max(a.partmax);
        if (threadIdx.x == 0) slam_new[0] = lam;
        for (int m = 0; m < a.M; ++m) {
            const double dtm = a.dt * a.dtau[m];
            const double* up = m ? Um((const double*)a.U, m - 1) : a.u0;
            const double* cp = m ? Um((const double*)a.CC, m - 1) : a.c0;
            double* um = Um(a.U, m);
            if (dtm != 0.0) {
                const double cimp = dtm * nut(dtm, lam);
                Terms t1{};
                t1.add(up, 1.0);
                t1.add(cp, dtm);
                if (!solve(um, up, t1, cimp)) return false;     // warm start u_{m-1}
                if (a.stages == 2) {
                    conv(um, CONV_OUT, a.tmpc, nullptr);
                    Terms t2{};
                    t2.add(up, 1.0);
                    t2.add(a.tmpc, dtm);
                    if (!solve(um, um, t2, cimp)) return false;
                }
            } else {
                Terms t0{};
                t0.add(up, 1.0);
                lin(um, t0);                               // Lobatto t_1 = t_0
                if (!bar()) return false;
            }
            conv(um, CONV_OUT, Um(a.CC, m), a.partmax + (size_t)(m + 1) * G);
            lap(um, Um(a.LU, m), Um(a.F, m), Um(a.CC, m));
            if (!bar()) return false;
            lam = total_max(a.partmax + (size_t)(m + 1) * G);
            if (threadIdx.x == 0) slam_new[m + 1] = lam;
        }
        __syncthreads();
        for (int t = threadIdx.x; t <= MMAX; t += blockDim.x) slam_old[t] = slam_new[t];
        __syncthreads();
        return true;
    }

    __device__ bool correct() {
        for (int k = 0; k < a.nsweeps; ++k) {
            quad();
            double lam = slam_old[0];                      // lam_max(u_0)
            for (int m = 0; m < a.M; ++m) {
                const double dtm = a.dt * a.dtau[m];
                const double* up = m ? Um((const double*)a.U, m - 1) : a.u0;
                double* um = Um(a.U, m);
                if (dtm == 0.0) {                          // Lobatto t_1 = t_0
                    Terms t{};
                    t.add(up, 1.0);
                    t.add(Um((const double*)a.Qb, m), 1.0);
                    if (a.G) t.add(Um(a.G, m), 1.0);
                    lin(um, t);
                    if (!bar()) return false;
                } else {
                    const double nu_new = nut(dtm, lam), nu_old = nut(dtm, slam_old[m]);
                    Terms t1{};
                    t1.add(up, 1.0);
                    t1.add(Um((const double*)a.Qb, m), 1.0);
                    if (a.G) t1.add(Um(a.G, m), 1.0);
                    t1.add(Um((const double*)a.LU, m), -dtm * nu_old);
                    Terms t2 = t1;
                    if (m > 0) t1.add(a.dC, dtm);          // c(u^k_{m-1}) - c(u^{k-1}_{m-1})
                    if (!solve(um, um, t1, dtm * nu_new)) return false;
                    if (a.stages == 2) {
                        conv(um, CONV_OUT, a.tmpc, nullptr);
                        t2.add(a.tmpc, dtm);               // c(u^(1))
                        t2.add(Um((const double*)a.CC, m), -dtm);   // c(u^{k-1}_m)
                        if (!solve(um, um, t2, dtm * nu_new)) return false;
                    }
                }
                conv(um, CONV_DELTA, Um(a.CC, m), a.partmax + (size_t)(m + 1) * G);
                lap(um, Um(a.LU, m), Um(a.F, m), Um(a.CC, m));
                if (!bar()) return false;
                lam = total_max(a.partmax + (size_t)(m + 1) * G);
                if (threadIdx.x == 0) slam_new[m + 1] = lam;
            }
            __syncthreads();
            for (int t = 1 + threadIdx.x; t <= MMAX; t += blockDim.x) slam_old[t] = slam_new[t];
            __syncthreads();
        }
        return true;
    }

    __device__ void finish() {
        __syncthreads();
        if (blockIdx.x == 0) {
            for (int t = threadIdx.x; t <= MMAX; t += blockDim.x) {
                a.lam[t] = slam_old[t];
                a.lam[MMAX + 1 + t] = slam_new[t];
            }
        }
    }
};

template <int NQ, int DIM, int PDE>
__global__ void __launch_bounds__(512, 1) k_sweep(const __grid_constant__ SweepArgs a) {
    Sweeper<NQ, DIM, PDE> s(a);
    bool ok;
    if (a.mode == SW_REFRESH) ok = s.refresh();
    else if (a.mode == SW_PREDICT) ok = s.predict();
    else ok = s.correct();
    if (ok) s.finish();
}

template <int NQ, int DIM, int PDE>
size_t sweep_smem(int epb) {
    using S = Sweeper<NQ, DIM, PDE>;
    return (2 * NQ * NQ + 3 * NQ + 32 + 2 * (MMAX + 1) + S::Q + (size_t)epb * S::NC * S::Q +
            (size_t)epb * S::NC * S::TRS + (size_t)epb * 2 * S::NC * S::Q) * sizeof(double);
}

template <int NQ, int DIM, int PDE>
int sweep_config_impl(const Geo& g, int* epb_out, int* block_out) {
    using S = Sweeper<NQ, DIM, PDE>;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int maxepb = S::Q >= 512 ? 1 : 512 / S::Q;
    long long want = (g.nel + nsm - 1) / nsm;      // aim at one tile per SM
    int epb = (int)(want < 1 ? 1 : (want > maxepb ? maxepb : want));
    const int minepb = (32 + S::Q - 1) / S::Q;     // at least one warp per block
    if (epb < minepb) epb = minepb > maxepb ? maxepb : minepb;
    const int bs = epb * S::Q;
    const size_t sh = sweep_smem<NQ, DIM, PDE>(epb);
    cudaFuncSetAttribute(k_sweep<NQ, DIM, PDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<NQ, DIM, PDE>, bs, sh) != cudaSuccess || per < 1)
        return 0;
    const long long ntiles = (g.nel + epb - 1) / epb;
    long long grid = (long long)per * nsm;
    if (grid > ntiles) grid = ntiles;
    *epb_out = epb;
    *block_out = bs;
    return (int)grid;
}

template <int NQ, int DIM, int PDE>
cudaError_t sweep_launch_impl(const SweepArgs& a, int grid, int block) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = sweep_smem<NQ, DIM, PDE>(a.epb);
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep<NQ, DIM, PDE>, a);
}

}  // namespace sisdc
