// Persistent cooperative SI-SDC sweep kernel (sm_103a).
//
// One launch runs a whole predictor sweep (eqs. sdc:incremental_predictor_si1
// and _si2), `nsweeps` incremental correction sweeps (Algorithm 1 with the
// SI(1)/SI(2) deltas, Sec. 3.3 and Sec. 4.3), or the cache refresh that makes
// f(U), c(U) and L U consistent with a new iterate.  Every block owns a fixed
// set of elements (all components) for the whole launch, so elementwise work
// (right-hand sides, the S.F quadrature, CG vector updates, f updates) needs
// no synchronisation; only neighbour coupling (face values of c(u), SIPG face
// lines) and global reductions (CG inner products, the largest spectral
// radius entering nu_tilde) go through the bounded grid barrier.  Data other
// blocks write during the launch is read through L2 (__ldcg).
//
// Operators: the SIPG application is one branch-free sum of products with
// pre-scaled coefficients (sipg.cuh); the Rusanov face fluxes of c(u) are
// evaluated once per face node in face tasks, x faces and y faces in
// separate whole warps, and added at the end nodes after a block barrier.
//
// Implicit solves: Jacobi-PCG on (M + c A) x = M b with two barriers per
// iteration.  The update phase stores z = D^-1 r beside r; a block forms the
// face lines of a neighbour's new search direction p_new = z + beta p_old
// itself, from the neighbour's z and p_old (p is double-buffered), with the
// same inline arithmetic the owner uses, so both sides of every face see
// bitwise-identical values and p never has to be published before use.
//
// MIX = true (mixed precision): the implicit solves run as an iterative
// refinement whose residual, right-hand side, inner products and solution
// update are FP64 while the inner CG (its matvecs and vectors) is FP32.  The
// explicit operator evaluations (c(u), L u) keep at least ~48-bit accuracy
// (FP64, or double-single arithmetic on the FP32 pipe for the scalar
// convection-diffusion and Burgers PDEs) and all cached quantities stay
// FP64: evaluated in FP32 they would perturb every sweep by eps_32 * dt_m *
// |c|, which the few sweeps of a step do not iterate away.
//
// The first residual of a solve whose initial guess is the previous iterate
// x0 = u^{k-1}_m reuses the cached L x0:  (M + c A) x0 = M x0 - c M L x0.
#pragma once
#include <type_traits>

#include "ops.h"
#include "ds.cuh"
#include "pde.cuh"
#include "sipg.cuh"

namespace sisdc {

template <int NQ, int DIM, int PDE, bool MIX>
struct Sweeper {
    using PD = Pde<PDE>;
    using RT = typename std::conditional<MIX, float, double>::type;   // operator arithmetic
    using CT = double;                                                 // cache storage (FP64)
    static constexpr int NC = PD::NC;
    static constexpr int NQY = DIM == 2 ? NQ : 1;
    static constexpr int Q = NQ * NQY;
    static constexpr int NF = 2 * DIM;
    static constexpr int TRS = NF * 2 * NQ;
    static constexpr int NCO = DIM * NQ + 4 * DIM;   // coefficients per node of the pre-scaled operator
    static constexpr int NTAB = NCO * Q + 4 * NQ;     // pre-scaled operator and face tables
    // arithmetic of the explicit operator evaluations (c(u), L u): FP64, or
    // double-single on the FP32 pipe in the mixed form of the scalar
    // convection-diffusion and Burgers PDEs
    static constexpr bool EXDS = MIX && (PDE == 0 || PDE == 1);
    using EX = typename std::conditional<EXDS, dsf, double>::type;

    // geometry factors in the arithmetic of the double-single evaluations
    struct GeoDS {
        dsf sx, sy, ihx, ihy, taux, tauy, hx, hy, liftLx, liftRx, liftLy, liftRy;
    };

    static size_t smem_bytes(int epb) {
        const size_t d = NTAB + 2 * NQ * NQ + 3 * NQ + 32 + 2 * (MMAX + 1) + Q   // tables, scratch, lam, dinv
                         + (size_t)epb * NC * Q + (size_t)epb * NC * TRS;         // FP64 tile + faces
        const size_t d2 = d + (size_t)epb * 2 * NC * Q;                          // FP64 fluxes
        size_t r = MIX ? (NTAB + 2 * NQ * NQ + 3 * NQ + Q + (size_t)epb * NC * Q + (size_t)epb * NC * TRS +
                          (size_t)epb * 2 * NC * Q)                                 // RT tables, tile, faces, fluxes
                       : 0;
        const size_t x = EXDS ? (2 * NQ * NQ + NQ + 16 + 4) : 0;          // double-single tables, geometry, params
        return d2 * sizeof(double) + r * sizeof(RT) + x * sizeof(dsf) + 16;
    }

    const SweepArgs& a;
    const Geo& g;
    PdeParams pp;
    PdeParamsT<dsf>* xpp;          // flux parameters in double-single (shared memory)
    GeoDS* xg;                     // geometry factors in double-single (shared memory)
    dsf *xD, *xK, *xw;             // D, K, w in double-single (shared memory)
    dsf imass_ds;                  // 1 / mass of the thread's node
    double *sA, *sDh, *sD, *sK, *sw, *sdx, *sdy, *scratch, *slam_old, *slam_new, *sdinv, *su, *sf, *sF64;
    RT *rA, *rDh, *rD, *rK, *rw, *rdx, *rdy, *rdinv, *ru, *rf, *sFR;
    int epb, le, node, i, j, G;
    long long ntiles, N, NV;
    double mass, imass, diagA;
    int solve_parity;
    int log_base, log_n;                  // solve-log slot of the next solve

    struct Terms {
        int n;
        const void* in[6];
        double cf[6];
        bool f32[6];
        __device__ void add(const double* p, double c) { in[n] = p; cf[n] = c; f32[n] = false; ++n; }
        __device__ void add(const float* p, double c) { in[n] = p; cf[n] = c; f32[n] = true; ++n; }
        __device__ double at(int q, long long id) const {
            return f32[q] ? (double)__ldcg((const float*)in[q] + id) : __ldcg((const double*)in[q] + id);
        }
    };

    __device__ CT* C(void* p) const { return static_cast<CT*>(p); }
    __device__ const CT* C(const void* p) const { return static_cast<const CT*>(p); }

    __device__ Sweeper(const SweepArgs& args) : a(args), g(args.g) {
        extern __shared__ double sm[];
        pp = PdeParams{a.gamma, a.ax, a.ay};
        epb = a.epb;
        sA = sm;                              // [NCO][Q] pre-scaled operator coefficients
        sDh = sA + NCO * Q;                   // [4][NQ] half-scaled face rows
        sD = sDh + 4 * NQ;
        sK = sD + NQ * NQ;
        sw = sK + NQ * NQ;
        sdx = sw + NQ;
        sdy = sdx + NQ;
        scratch = sdy + NQ;
        slam_old = scratch + 32;
        slam_new = slam_old + MMAX + 1;
        sdinv = slam_new + MMAX + 1;
        su = sdinv + Q;                       // [epb][NC][Q] FP64 tile
        sf = su + epb * NC * Q;               // [epb][NC][NF][2][NQ] FP64 faces
        sF64 = sf + epb * NC * TRS;           // [epb][2][NC][Q] FP64 fluxes
        RT* rbase = reinterpret_cast<RT*>(sF64 + epb * 2 * NC * Q);
        if (MIX) {
            rA = rbase;
            rDh = rA + NCO * Q;
            rD = rDh + 4 * NQ;
            rK = rD + NQ * NQ;
            rw = rK + NQ * NQ;
            rdx = rw + NQ;
            rdy = rdx + NQ;
            rdinv = rdy + NQ;
            ru = rdinv + Q;
            rf = ru + epb * NC * Q;
            sFR = rf + epb * NC * TRS;
        } else {
            rA = reinterpret_cast<RT*>(sA);
            rDh = reinterpret_cast<RT*>(sDh);
            rD = reinterpret_cast<RT*>(sD);
            rK = reinterpret_cast<RT*>(sK);
            rw = reinterpret_cast<RT*>(sw);
            rdx = reinterpret_cast<RT*>(sdx);
            rdy = reinterpret_cast<RT*>(sdy);
            rdinv = reinterpret_cast<RT*>(sdinv);
            ru = reinterpret_cast<RT*>(su);
            rf = reinterpret_cast<RT*>(sf);
            sFR = reinterpret_cast<RT*>(sF64);
        }
        if constexpr (EXDS) {
            const size_t rcount = NTAB + 2 * NQ * NQ + 3 * NQ + Q + (size_t)epb * NC * Q +
                                  (size_t)epb * NC * TRS + (size_t)epb * 2 * NC * Q;
            xD = reinterpret_cast<dsf*>(rbase + ((rcount + 1) & ~size_t(1)));
            xK = xD + NQ * NQ;
            xw = xK + NQ * NQ;
            xg = reinterpret_cast<GeoDS*>(xw + NQ);
            xpp = reinterpret_cast<PdeParamsT<dsf>*>(xg + 1);
            if (threadIdx.x == 0) {
                *xg = GeoDS{dsf(g.sx), dsf(g.sy), dsf(g.ihx), dsf(g.ihy), dsf(g.taux), dsf(g.tauy),
                            dsf(g.hx), dsf(g.hy), dsf(g.liftLx), dsf(g.liftRx), dsf(g.liftLy), dsf(g.liftRy)};
                *xpp = PdeParamsT<dsf>{dsf(a.gamma), dsf(a.ax), dsf(a.ay)};
            }
        }
        for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
            sD[t] = g.D[t];
            sK[t] = g.K[t];
            if (MIX) {
                rD[t] = (RT)g.D[t];
                rK[t] = (RT)g.K[t];
            }
            if constexpr (EXDS) {
                xD[t] = dsf(g.D[t]);
                xK[t] = dsf(g.K[t]);
            }
        }
        for (int t = threadIdx.x; t < NQ; t += blockDim.x) {
            sw[t] = g.w[t];
            sdx[t] = g.dline_x[t];
            sdy[t] = g.dline_y[t];
            if (MIX) {
                rw[t] = (RT)g.w[t];
                rdx[t] = (RT)g.dline_x[t];
                rdy[t] = (RT)g.dline_y[t];
            }
            if constexpr (EXDS) xw[t] = dsf(g.w[t]);
        }
        for (int t = threadIdx.x; t < NCO * Q; t += blockDim.x) {
            const int k = t / Q, nd = t - k * Q;
            const double v = sipg_opA_coeff<NQ, DIM>(g, g.D, g.K, g.w, k, nd % NQ, nd / NQ);
            sA[t] = v;
            if (MIX) rA[t] = (RT)v;
        }
        for (int t = threadIdx.x; t < 4 * NQ; t += blockDim.x) {
            const int f = t / NQ, q = t - f * NQ;
            const double v = 0.5 * (f < 2 ? g.sx : g.sy) * g.D[((f & 1) ? NQ - 1 : 0) * NQ + q];
            sDh[t] = v;
            if (MIX) rDh[t] = (RT)v;
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
        NV = (long long)NC * N;
        solve_parity = 0;
        log_base = a.log_count ? __ldcg(a.log_count) : 0;
        log_n = 0;
        __syncthreads();
        mass_diag(i, j, mass, diagA);
        imass = 1.0 / mass;
        if constexpr (EXDS) imass_ds = dsf(imass);
    }

    // geometry factors, flux parameters and operator tables in arithmetic V
    template <class V>
    __device__ const auto& geo() const {
        if constexpr (std::is_same<V, dsf>::value) return *xg;
        else return g;
    }
    template <class V>
    __device__ const auto& par() const {
        if constexpr (std::is_same<V, dsf>::value) return *xpp;
        else return pp;
    }
    template <class V>
    __device__ const V* tab_D() const {
        if constexpr (std::is_same<V, double>::value) return sD;
        else if constexpr (std::is_same<V, dsf>::value) return xD;
        else return reinterpret_cast<const V*>(rD);
    }
    template <class V>
    __device__ const V* tab_A() const {
        if constexpr (std::is_same<V, double>::value) return sA;
        else return reinterpret_cast<const V*>(rA);
    }
    template <class V>
    __device__ const V* tab_Dh() const {
        if constexpr (std::is_same<V, double>::value) return sDh;
        else return reinterpret_cast<const V*>(rDh);
    }
    template <class V>
    __device__ const V* tab_K() const {
        if constexpr (std::is_same<V, double>::value) return sK;
        else if constexpr (std::is_same<V, dsf>::value) return xK;
        else return reinterpret_cast<const V*>(rK);
    }
    template <class V>
    __device__ const V* tab_w() const {
        if constexpr (std::is_same<V, double>::value) return sw;
        else if constexpr (std::is_same<V, dsf>::value) return xw;
        else return reinterpret_cast<const V*>(rw);
    }
    // tile, face and flux buffers: the FP32 ones for V = float, else the
    // 8-byte ones (double and double-single have the same size)
    template <class V>
    __device__ V* buf_tile() const {
        return std::is_same<V, float>::value ? reinterpret_cast<V*>(ru) : reinterpret_cast<V*>(su);
    }
    template <class V>
    __device__ V* buf_face() const {
        return std::is_same<V, float>::value ? reinterpret_cast<V*>(rf) : reinterpret_cast<V*>(sf);
    }
    template <class V>
    __device__ V* buf_flux() const {
        return std::is_same<V, float>::value ? reinterpret_cast<V*>(sFR) : reinterpret_cast<V*>(sF64);
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

    __device__ bool bar() { return grid_barrier(a.bar_count, a.bar_exit, a.err); }

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

    // run f(e0, nle) over the block's element tiles
    template <class F>
    __device__ void tiles(F f) {
        for (long long t = blockIdx.x; t < ntiles; t += G) {
            const long long e0 = t * epb;
            f(e0, (int)min((long long)epb, (long long)g.nel - e0));
        }
    }

    __device__ long long vidx(int c, long long e) const { return c * N + e * Q + node; }

    __device__ long long neighbour(long long e, int f) const {
        // element counts are capped at 2^30, so 32-bit division suffices
        const int ei = (int)e, ey = ei / g.nex, ex = ei - ey * g.nex;
        if (f == 0) return (long long)(ei + (ex == 0 ? g.nex - 1 : -1));
        if (f == 1) return (long long)(ei + (ex == g.nex - 1 ? 1 - g.nex : 1));
        if (f == 2) return (long long)(ey == 0 ? ei + (g.ney - 1) * g.nex : ei - g.nex);
        return (long long)(ey == g.ney - 1 ? ex : ei + g.nex);
    }

    // node of the line normal to face f through face row k, position q
    __device__ static int line_node(int f, int k, int q) { return f < 2 ? k * NQ + q : q * NQ + k; }

    // ---- SIPG face terms and operator, in arithmetic V ------------------------
    // jumps [u] and averages {u'} on the faces of the tile's elements: own
    // lines from the tile tu, neighbour lines from getv(c, e, node).
    template <class V, class GetV>
    __device__ void faces(int nle, long long e0, const V* tu, V* tf, const V* Dt, GetV getv) {
        const int per = NC * NF * NQ;
        for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
            const int l = t / per;
            int rem = t - l * per;
            const int c = rem / (NF * NQ);
            rem -= c * NF * NQ;
            const int f = rem / NQ, k = rem - f * NQ;
            if (f < 2 && k >= NQY) continue;
            const long long en = neighbour(e0 + l, f);
            const V* u = tu + (l * NC + c) * Q;
            V vo[NQ], vn[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                vo[q] = u[line_node(f, k, q)];
                vn[q] = getv(c, en, line_node(f ^ 1, k, q));
            }
            V jump, avg;
            if constexpr (std::is_same<V, dsf>::value) sipg_face<NQ>(geo<V>(), vo, vn, f, Dt, jump, avg);
            else sipg_face_pre<NQ>(vo, vn, f, tab_Dh<V>(), jump, avg);
            V* o = tf + ((l * NC + c) * NF + f) * 2 * NQ;
            o[k] = jump;
            o[NQ + k] = avg;
        }
    }

    // (A u)(i, j) for component c of local element l
    template <class V>
    __device__ V opA(int l, int c, const V* tu, const V* tf, const V* Dt, const V* Kt, const V* wt) const {
        if constexpr (std::is_same<V, dsf>::value)
            return sipg_opA<NQ, DIM, V>(geo<V>(), i, j, tu + (l * NC + c) * Q, tf + (l * NC + c) * TRS, Dt, Kt, wt);
        else
            return sipg_opA_pre<NQ, DIM, V>(i, j, tu + (l * NC + c) * Q, tf + (l * NC + c) * TRS, tab_A<V>() + node);
    }
    __device__ double opA64(int l, int c) const { return opA<double>(l, c, su, sf, sD, sK, sw); }
    __device__ RT opAR(int l, int c) const { return opA<RT>(l, c, ru, rf, rD, rK, rw); }

    // new search direction from the stored z = D^-1 r (shared by owner and neighbours)
    __device__ static double znew(double z, double beta, double pold) { return beta == 0.0 ? z : z + beta * pold; }

    // new search direction at one node (shared by owner and neighbours)
    template <class V>
    __device__ static V pnew(V r, V dinv, V beta, V pold) {
        const V z = r * dinv;
        return beta == V(0) ? z : z + beta * pold;
    }

    __device__ void set_dinv(double c) {
        __syncthreads();
        for (int t = threadIdx.x; t < Q; t += blockDim.x) {
            double ms, dg;
            mass_diag(t % NQ, t / NQ, ms, dg);
            sdinv[t] = 1.0 / (ms + c * dg);
            if (MIX) rdinv[t] = (RT)sdinv[t];
        }
        __syncthreads();
    }

    __device__ void stat_solve(int it, bool fin, bool conv_ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (a.iters_out) *a.iters_out += it;
            atomicAdd((unsigned long long*)&a.stats[ST_SOLVES], 1ull);
            atomicAdd((unsigned long long*)&a.stats[ST_ITERS], (unsigned long long)it);
            atomicMax((unsigned long long*)&a.stats[ST_MAXIT], (unsigned long long)it);
            if (!fin) {
                atomicOr(a.err, DEV_NONFINITE);
            } else if (!conv_ok) {
                atomicOr(a.err, DEV_NOCONV);
                atomicAdd((unsigned long long*)&a.stats[ST_NOCONV], 1ull);
            }
        }
    }

    // ---- implicit solve (FP64) ---------------------------------------------------
    // (M + c A) x = M b, b = sum_t cf_t in_t.  The initial guess is xsrc (x
    // itself when xsrc == x); neighbours' xsrc must be final on entry.
    __device__ bool solve64(double* x, const double* xsrc, const Terms& tm, double c, const double* Lx0) {
        double* part = a.part + (size_t)(solve_parity ? 8 : 0) * G;
        solve_parity ^= 1;
        set_dinv(c);
        const double dinv = sdinv[node];
        double acc_bb = 0.0, acc = 0.0;
        // preconditioned residual z = D^-1 r, stored with r so that a search
        // direction p = z + beta p_old costs one FMA for owner and neighbours
        double* Z = static_cast<double*>(a.rf);
        const int slot = log_base + log_n;
        const bool logit = a.log_r && slot < a.log_cap;
        ++log_n;
        double* lr = logit ? a.log_r + (long long)slot * NV : nullptr;
        double* ldx = logit ? a.log_dx + (long long)slot * NV : nullptr;
        if (logit && blockIdx.x == 0 && threadIdx.x == 0) a.log_c[slot] = c;
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
            if (!Lx0)
                faces<double>(nle, e0, su, sf, sD, [&](int cc, long long en, int nd) { return __ldcg(xsrc + cc * N + en * Q + nd); });
            __syncthreads();
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    double b = 0.0;
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        if (q < tm.n) b += tm.cf[q] * tm.at(q, id);
                    const double mb = mass * b;
                    const double xv = su[(le * NC + cc) * Q + node];
                    const double Ax = Lx0 ? -mass * __ldcg(Lx0 + id) : opA64(le, cc);
                    const double rr = mb - (mass * xv + c * Ax);
                    const double zz = rr * dinv;
                    a.r[id] = rr;
                    Z[id] = zz;
                    if (logit) {
                        lr[id] = rr / mass;      // nodal residual b - (x0 - c L x0)
                        ldx[id] = xv;
                    }
                    acc_bb += mb * mb * dinv;
                    acc += rr * zz;
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
        double* P0 = static_cast<double*>(a.p);
        double* P1 = static_cast<double*>(a.p2);
        double* AP = static_cast<double*>(a.Ap);
        while (fin && rz > tol2 && it < a.maxit) {
            const double* pold = par ? P1 : P0;
            double* pcur = par ? P0 : P1;
            acc = 0.0;
            tiles([&](const long long e0, const int nle) {
                const bool act = le < nle;
                const long long e = e0 + le;
                double pn[NC];
                if (act) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e);
                        pn[cc] = znew(__ldcg(Z + id), beta, beta == 0.0 ? 0.0 : __ldcg(pold + id));
                        pcur[id] = pn[cc];
                        su[(le * NC + cc) * Q + node] = pn[cc];
                    }
                }
                __syncthreads();
                faces<double>(nle, e0, su, sf, sD, [&](int cc, long long en, int nd) {
                    const long long id = cc * N + en * Q + nd;
                    return znew(__ldcg(Z + id), beta, beta == 0.0 ? 0.0 : __ldcg(pold + id));
                });
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const double Apv = mass * pn[cc] + c * opA64(le, cc);
                        AP[vidx(cc, e)] = Apv;
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
                        const double rr = __ldcg(a.r + id) - alpha * __ldcg(AP + id);
                        const double zz = rr * dinv;
                        a.r[id] = rr;
                        Z[id] = zz;
                        acc += rr * zz;
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
        if (logit) {
            tiles([&](const long long e0, const int nle) {
                if (le < nle) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e0 + le);
                        ldx[id] = __ldcg(x + id) - __ldcg(ldx + id);
                    }
                }
            });
        }
        stat_solve(it, fin, !(rz > tol2));
        return true;
    }

    // ---- implicit solve (mixed: FP64 refinement residual, FP32 inner PCG) --------
    // Outer iterative refinement in FP64: r = M b - (M + c A) x with the FP64
    // operator; inner Jacobi-PCG in FP32 on (M + c A) d = r from d = 0 with
    // FP64-accumulated inner products; x += d accumulated in FP64.  Stops when
    // the FP64 residual meets the same criterion as the FP64 solve.
    __device__ bool solve_mix(double* x, const double* xsrc, const Terms& tm, double c, const double* Lx0) {
        double* part = a.part + (size_t)(solve_parity ? 8 : 0) * G;
        solve_parity ^= 1;
        set_dinv(c);
        const double dinv = sdinv[node];
        const RT dinvr = rdinv[node];
        const RT cr = (RT)c, massr = (RT)mass;
        RT* RF = static_cast<RT*>(a.rf);
        RT* P0 = static_cast<RT*>(a.p);
        RT* P1 = static_cast<RT*>(a.p2);
        RT* AP = static_cast<RT*>(a.Ap);
        double bb = 0.0, tol2 = 0.0;
        bool fin = true, done = false;
        int its = 0, ir = 0;
        const int max_ir = 30;
        for (; ir < max_ir; ++ir) {
            // FP64 refinement residual (first pass also forms M b and copies xsrc)
            const double* xs = ir == 0 ? xsrc : x;
            double acc_bb = 0.0, acc64 = 0.0, acc32 = 0.0;
            tiles([&](const long long e0, const int nle) {
                const bool act = le < nle;
                const long long e = e0 + le;
                if (act) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e);
                        const double xv = __ldcg(xs + id);
                        su[(le * NC + cc) * Q + node] = xv;
                        if (ir == 0 && xsrc != x) x[id] = xv;
                    }
                }
                __syncthreads();
                if (!(ir == 0 && Lx0))
                    faces<double>(nle, e0, su, sf, sD, [&](int cc, long long en, int nd) { return __ldcg(xs + cc * N + en * Q + nd); });
                __syncthreads();
                if (act) {
                    RT loc32 = RT(0);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        const long long id = vidx(cc, e);
                        double mb;
                        if (ir == 0) {
                            double b = 0.0;
#pragma unroll
                            for (int q = 0; q < 6; ++q)
                                if (q < tm.n) b += tm.cf[q] * tm.at(q, id);
                            mb = mass * b;
                            a.r[id] = mb;
                            acc_bb += mb * mb * dinv;
                        } else {
                            mb = __ldcg(a.r + id);
                        }
                        const double xv = su[(le * NC + cc) * Q + node];
                        const double Ax = (ir == 0 && Lx0) ? -mass * __ldcg(Lx0 + id) : opA64(le, cc);
                        const double r64 = mb - (mass * xv + c * Ax);
                        acc64 += r64 * (r64 * dinv);
                        const RT r32 = to_v<RT>(r64);
                        RF[id] = r32;
                        loc32 += r32 * (r32 * dinvr);
                    }
                    acc32 += to_f64(loc32);
                }
                __syncthreads();
            });
            if (ir == 0) put_partial(part, acc_bb);
            put_partial(part + G, acc64);
            put_partial(part + 2 * G, acc32);
            if (!bar()) return false;
            if (ir == 0) {
                bb = total(part);
                tol2 = fmax(a.rtol * a.rtol * bb, 1e-300);
            }
            const double rz64 = total(part + G);
            double rz = total(part + 2 * G);
            fin = isfinite(rz64) && isfinite(bb);
            if (!fin || !(rz64 > tol2)) {
                done = fin;
                break;
            }
            // inner FP32 PCG from d = 0 (x += alpha p applied to x directly)
            const double tol_in = fmax(1e-10 * rz, 0.25 * tol2);
            int par = 0;
            double beta = 0.0;
            while (rz > tol_in && its < a.maxit) {
                const RT* pold = par ? P1 : P0;
                RT* pcur = par ? P0 : P1;
                const RT betar = (RT)beta;
                double acc = 0.0;
                tiles([&](const long long e0, const int nle) {
                    const bool act = le < nle;
                    const long long e = e0 + le;
                    RT pn[NC];
                    if (act) {
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            const long long id = vidx(cc, e);
                            pn[cc] = pnew<RT>(__ldcg(RF + id), dinvr, betar, betar == RT(0) ? RT(0) : __ldcg(pold + id));
                            pcur[id] = pn[cc];
                            ru[(le * NC + cc) * Q + node] = pn[cc];
                        }
                    }
                    __syncthreads();
                    faces<RT>(nle, e0, ru, rf, rD, [&](int cc, long long en, int nd) {
                        const long long id = cc * N + en * Q + nd;
                        return pnew<RT>(__ldcg(RF + id), rdinv[nd], betar, betar == RT(0) ? RT(0) : __ldcg(pold + id));
                    });
                    __syncthreads();
                    if (act) {
                        // the thread's products in FP32, one conversion, FP64 accumulation
                        // over threads and blocks (FP32<->FP64 conversions use the FP64 pipe)
                        RT loc = RT(0);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            const RT Apv = massr * pn[cc] + cr * opAR(le, cc);
                            AP[vidx(cc, e)] = Apv;
                            loc += pn[cc] * Apv;
                        }
                        acc += to_f64(loc);
                    }
                    __syncthreads();
                });
                put_partial(part + 3 * G, acc);
                if (!bar()) return false;
                const double alpha = rz / total(part + 3 * G);
                const RT alphar = (RT)alpha;
                acc = 0.0;
                tiles([&](const long long e0, const int nle) {
                    if (le < nle) {
                        const long long e = e0 + le;
                        RT loc = RT(0);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            const long long id = vidx(cc, e);
                            x[id] = __ldcg(x + id) + alpha * to_f64(__ldcg(pcur + id));
                            const RT rr = __ldcg(RF + id) - alphar * __ldcg(AP + id);
                            RF[id] = rr;
                            loc += rr * (rr * dinvr);
                        }
                        acc += to_f64(loc);
                    }
                });
                put_partial(part + 4 * G, acc);
                if (!bar()) return false;
                const double rzn = total(part + 4 * G);
                beta = rzn / rz;
                rz = rzn;
                ++its;
                par ^= 1;
                if (!isfinite(rz)) break;
            }
            if (its >= a.maxit) break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0)
            atomicAdd((unsigned long long*)&a.stats[ST_IR], (unsigned long long)(ir + 1));
        stat_solve(its, fin, done);
        return true;
    }

    // Lx0 (nullable): cached L xsrc, which replaces the first matvec
    __device__ bool solve(double* x, const double* xsrc, const Terms& tm, double c, const double* Lx0 = nullptr) {
        if (MIX) return solve_mix(x, xsrc, tm, c, Lx0);
        return solve64(x, xsrc, tm, c, Lx0);
    }

    // One face node of the convective operator, for local element l, face
    // side (0: left/lower, 1: right/upper) of direction x (XD) or y, face row
    // k: stores the lifted difference between the Rusanov flux and the own
    // normal flux, the correction of c(u) at the own end node, in the face
    // buffer tf ([l][c][f][k]); Navier-Stokes with visc: also the BR1
    // correction of the gradient of w = (v_x, v_y, T) at that node, lift
    // times ({w} - w) with the central trace {w} ([l][q][NF + f][k]).
    template <class V, bool XD>
    __device__ void conv_face(const double* X, int l, long long e0, int side, int k, bool visc, V* tf) const {
        const auto& gv = geo<V>();
        const auto& pv = par<V>();
        const int f = (XD ? 0 : 2) + side;
        const int io = side ? NQ - 1 : 0, in = NQ - 1 - io;
        const int nd = XD ? k * NQ + io : io * NQ + k;
        const int ndn = XD ? k * NQ + in : in * NQ + k;
        const long long e = e0 + l, en = neighbour(e, f);
        V uo[NC], un[NC], d[NC];
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            uo[cc] = to_v<V>(__ldcg(X + cc * N + e * Q + nd));
            un[cc] = to_v<V>(__ldcg(X + cc * N + en * Q + ndn));
        }
        rusanov_jump<PDE, XD>(pv, uo, un, side == 1, d);
        // c(u) gains +liftL (Fs - F) at a left end node, -liftR (Fs - F) at a right one
        const V lift = XD ? (side ? -V(gv.liftRx) : V(gv.liftLx)) : (side ? -V(gv.liftRy) : V(gv.liftLy));
        V* o = tf + (size_t)l * NC * TRS + f * NQ + k;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) o[cc * TRS] = lift * d[cc];
        if constexpr (PD::VISC) {
            if (visc) {
                V wo[3], wn[3];
                PD::primitive(pv, uo, wo);
                PD::primitive(pv, un, wn);
#pragma unroll
                for (int q = 0; q < 3; ++q) o[q * TRS + NF * NQ] = -lift * (V(0.5) * (wo[q] + wn[q]) - wo[q]);
            }
        }
    }

    // ---- convective operator phase (arithmetic V) ------------------------------
    // c(X) for the block's elements into out (CT); mode CONV_DELTA also
    // writes dC = c - out_old; f64 (optional) receives c in FP64 (the start of
    // the cached f); optional spectral-radius partial into lamslot.
    // Navier-Stokes with f64 given: also the BR1 lifted gradients of the
    // primitive variables w = (v_x, v_y, T) (central traces {w}) and the
    // viscous flux from them, into a.FV; its divergence is added to f by lap().
    template <class V>
    __device__ void conv(const double* X, int mode, CT* out, double* f64, double* lamslot) {
        V* sFv = buf_flux<V>();
        V* tf = buf_face<V>();
        const V* Dv = tab_D<V>();
        const auto& gv = geo<V>();
        const auto& pv = par<V>();
        const bool visc = PD::VISC && f64 != nullptr;
        double lmax = 0.0;
        tiles([&](const long long e0, const int nle) {
            const bool act = le < nle;
            const long long e = e0 + le;
            V u[NC], Fx[NC], Fy[NC];
            V* sFx = sFv + (size_t)le * 2 * NC * Q;
            V* sFy = sFx + NC * Q;
            V w[3], gx[3], gy[3];
            V* sW = reinterpret_cast<V*>(su) + (size_t)le * NC * Q;    // primitive values (tile buffer is free here)
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) u[cc] = to_v<V>(__ldcg(X + vidx(cc, e)));
                if constexpr (PD::VISC) {
                    if (visc) {
                        PD::primitive(pv, u, w);
#pragma unroll
                        for (int k = 0; k < 3; ++k) sW[k * Q + node] = w[k];
                    }
                }
                PD::fx(pv, u, Fx);
                lmax = fmax(lmax, to_f64(PD::rx(pv, u)));
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) sFx[cc * Q + node] = Fx[cc];
                if (DIM == 2) {
                    PD::fy(pv, u, Fy);
                    lmax = fmax(lmax, to_f64(PD::ry(pv, u)));
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) sFy[cc * Q + node] = Fy[cc];
                }
            }
            // face tasks, one per face node, x faces first (padded to whole
            // warps so that each warp evaluates one flux direction)
            {
                const int nx = nle * 2 * NQY, xr = (nx + 31) & ~31;
                const int ny = DIM == 2 ? nle * 2 * NQ : 0;
                for (int t = threadIdx.x; t < xr + ny; t += blockDim.x) {
                    if (t < nx) {
                        const int l = t / (2 * NQY), r = t - l * 2 * NQY;
                        conv_face<V, true>(X, l, e0, r / NQY, r % NQY, visc, tf);
                    } else if (t >= xr) {
                        const int ty = t - xr, l = ty / (2 * NQ), r = ty - l * 2 * NQ;
                        conv_face<V, false>(X, l, e0, r / NQ, r % NQ, visc, tf);
                    }
                }
            }
            __syncthreads();
            if (act) {
                V cv[NC];
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    V s = V(0);
#pragma unroll
                    for (int k = 0; k < NQ; ++k) s += Dv[i * NQ + k] * sFx[cc * Q + j * NQ + k];
                    cv[cc] = -V(gv.sx) * s;
                }
                if (DIM == 2) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        V s = V(0);
#pragma unroll
                        for (int k = 0; k < NQ; ++k) s += Dv[j * NQ + k] * sFy[cc * Q + k * NQ + i];
                        cv[cc] -= V(gv.sy) * s;
                    }
                }
                if constexpr (PD::VISC) {
                    if (visc) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            V s = V(0), t = V(0);
#pragma unroll
                            for (int k = 0; k < NQ; ++k) {
                                s += Dv[i * NQ + k] * sW[q * Q + j * NQ + k];
                                t += Dv[j * NQ + k] * sW[q * Q + k * NQ + i];
                            }
                            gx[q] = V(gv.sx) * s;
                            gy[q] = V(gv.sy) * t;
                        }
                    }
                }
                // face corrections of the end nodes (conv_face)
                const V* fc = tf + (size_t)le * NC * TRS;
                auto add_face = [&](int f, int k) {
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) cv[cc] += fc[cc * TRS + f * NQ + k];
                    if constexpr (PD::VISC) {
                        if (visc) {
                            V* gd = f < 2 ? gx : gy;
#pragma unroll
                            for (int q = 0; q < 3; ++q) gd[q] += fc[q * TRS + NF * NQ + f * NQ + k];
                        }
                    }
                };
                if (i == 0) add_face(0, j);
                if (i == NQ - 1) add_face(1, j);
                if (DIM == 2) {
                    if (j == 0) add_face(2, i);
                    if (j == NQ - 1) add_face(3, i);
                }
                if constexpr (PD::VISC) {
                    if (visc) {
                        V fx[3], fy[3];
                        PD::vflux(V(a.mu), V(a.kappa), w, gx, gy, fx, fy);
                        const long long id0 = e * Q + node;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            a.FV[q * N + id0] = (double)fx[q];
                            a.FV[(3 + q) * N + id0] = (double)fy[q];
                        }
                    }
                }
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    const double cvd = to_f64(cv[cc]);
                    if (mode == CONV_DELTA) C(a.dC)[id] = cvd - __ldcg(out + id);
                    out[id] = cvd;
                    if (f64) f64[id] = cvd;
                }
            }
            __syncthreads();
        });
        if (lamslot) put_partial_max(lamslot, lmax);
    }

    // LU = L X (arithmetic V, stored CT); F += nu LU in FP64, F holding c(X)
    // from the conv phase of the same block (neighbours' X must be final)
    template <class V>
    __device__ void lap(const double* X, CT* LUm, double* Fm) {
        V* tu = buf_tile<V>();
        V* tf = buf_face<V>();
        const V* Dv = tab_D<V>();
        const V* Kv = tab_K<V>();
        const V* wv = tab_w<V>();
        tiles([&](const long long e0, const int nle) {
            const bool act = le < nle;
            const long long e = e0 + le;
            double* sV = sF64 + (size_t)le * 6 * Q;     // own viscous fluxes (Navier-Stokes)
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) tu[(le * NC + cc) * Q + node] = to_v<V>(__ldcg(X + vidx(cc, e)));
                if constexpr (PD::VISC)
#pragma unroll
                    for (int q = 0; q < 6; ++q) sV[q * Q + node] = __ldcg(a.FV + q * N + e * Q + node);
            }
            __syncthreads();
            faces<V>(nle, e0, tu, tf, Dv, [&](int cc, long long en, int nd) { return to_v<V>(__ldcg(X + cc * N + en * Q + nd)); });
            __syncthreads();
            if (act) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    V lu;
                    if constexpr (std::is_same<V, dsf>::value) lu = -(opA<V>(le, cc, tu, tf, Dv, Kv, wv) * imass_ds);
                    else lu = -opA<V>(le, cc, tu, tf, Dv, Kv, wv) * (V)imass;
                    const double lud = to_f64(lu);
                    LUm[id] = lud;
                    Fm[id] = __ldcg(Fm + id) + a.nu * lud;
                }
                if constexpr (PD::VISC) {
                    // div F_v with central face fluxes: (2/h) D F_v plus
                    // +- lift ({F_v} - F_v) at the end nodes (BR1)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        double s = 0.0, t = 0.0;
#pragma unroll
                        for (int k = 0; k < NQ; ++k) {
                            s += sD[i * NQ + k] * sV[q * Q + j * NQ + k];
                            t += sD[j * NQ + k] * sV[(3 + q) * Q + k * NQ + i];
                        }
                        double dx = g.sx * s, dy = g.sy * t;
                        const double fx = sV[q * Q + node], fy = sV[(3 + q) * Q + node];
                        if (i == NQ - 1) {
                            const double nb = __ldcg(a.FV + q * N + neighbour(e, 1) * Q + j * NQ);
                            dx += g.liftRx * (0.5 * (fx + nb) - fx);
                        }
                        if (i == 0) {
                            const double nb = __ldcg(a.FV + q * N + neighbour(e, 0) * Q + j * NQ + NQ - 1);
                            dx += -g.liftLx * (0.5 * (fx + nb) - fx);
                        }
                        if (j == NQ - 1) {
                            const double nb = __ldcg(a.FV + (3 + q) * N + neighbour(e, 3) * Q + i);
                            dy += g.liftRy * (0.5 * (fy + nb) - fy);
                        }
                        if (j == 0) {
                            const double nb = __ldcg(a.FV + (3 + q) * N + neighbour(e, 2) * Q + (NQ - 1) * NQ + i);
                            dy += -g.liftLy * (0.5 * (fy + nb) - fy);
                        }
                        const long long id = vidx(1 + q, e);
                        Fm[id] = __ldcg(Fm + id) + (dx + dy);
                    }
                }
            }
            __syncthreads();
        });
    }

    // elementwise: out = sum_t cf_t in_t over the block's nodes (FP64)
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
                        if (q < tm.n) v += tm.cf[q] * tm.at(q, id);
                    out[id] = v;
                }
            }
        });
    }

    // elementwise S.F quadrature Q_m = dt sum_i W[m][i] F_i (FP64 accumulation)
    __device__ void quad() {
        const double* F = a.F;
        tiles([&](const long long e0, const int nle) {
            if (le < nle) {
                const long long e = e0 + le;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const long long id = vidx(cc, e);
                    double f[MMAX];
#pragma unroll
                    for (int q = 0; q < MMAX; ++q) f[q] = q < a.M ? (double)__ldcg(F + q * NV + id) : 0.0;
#pragma unroll
                    for (int m = 0; m < MMAX; ++m) {
                        if (m >= a.M) break;
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < MMAX; ++q)
                            if (q < a.M) s += a.W[m * a.M + q] * f[q];
                        a.Qb[m * NV + id] = a.dt * s;
                    }
                }
            }
        });
    }

    __device__ double nut(double dtm, double lam) const {
        return a.nu_tilde_fix > 0.0 ? a.nu_tilde_fix : a.nu_d + a.nu_lam * lam + 0.5 * dtm * lam * lam;
    }
    __device__ double* Um(double* U, int m) const { return U + (long long)m * NV; }
    __device__ const double* Um(const double* U, int m) const { return U + (long long)m * NV; }
    __device__ CT* Cm(void* A, int m) const { return C(A) + (long long)m * NV; }

    // ---- the three modes ------------------------------------------------------
    // Navier-Stokes: the viscous divergence of lap() reads the neighbours'
    // viscous fluxes of the preceding conv(), and the next conv() overwrites
    // them: both need a grid barrier.
    __device__ bool visc_bar() { return PD::VISC ? bar() : true; }

    __device__ bool feval() {
        conv<EX>(a.u0, CONV_OUT, C(a.tmpc), a.fout, nullptr);
        if (!visc_bar()) return false;
        lap<EX>(a.u0, C(a.dC), a.fout);
        return true;
    }

    __device__ bool refresh() {
        conv<EX>(a.u0, CONV_OUT, C(a.c0), nullptr, a.partmax);
        for (int m = 0; m < a.M; ++m) {
            conv<EX>(Um(a.U, m), CONV_OUT, Cm(a.CC, m), Um(a.F, m), a.partmax + (size_t)(m + 1) * G);
            if (!visc_bar()) return false;
            lap<EX>(Um(a.U, m), Cm(a.LU, m), Um(a.F, m));
            if (!visc_bar()) return false;
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
        conv<EX>(a.u0, CONV_OUT, C(a.c0), nullptr, a.partmax);
        if (!bar()) return false;
        double lam = total_max(a.partmax);
        if (threadIdx.x == 0) slam_new[0] = lam;
        for (int m = 0; m < a.M; ++m) {
            const double dtm = a.dt * a.dtau[m];
            const double* up = m ? Um((const double*)a.U, m - 1) : a.u0;
            const CT* cp = m ? Cm(a.CC, m - 1) : C((const void*)a.c0);
            double* um = Um(a.U, m);
            if (dtm != 0.0) {
                const double cimp = dtm * nut(dtm, lam);
                Terms t1{};
                t1.add(up, 1.0);
                t1.add(cp, dtm);
                if (!solve(um, up, t1, cimp, m ? Cm(a.LU, m - 1) : nullptr)) return false;   // warm start u_{m-1}
                if (a.stages == 2) {
                    conv<EX>(um, CONV_OUT, C(a.tmpc), nullptr, nullptr);
                    Terms t2{};
                    t2.add(up, 1.0);
                    t2.add((const CT*)C(a.tmpc), dtm);
                    if (!solve(um, um, t2, cimp)) return false;
                }
            } else {
                Terms t0{};
                t0.add(up, 1.0);
                lin(um, t0);                               // Lobatto t_1 = t_0
                if (!bar()) return false;
            }
            conv<EX>(um, CONV_OUT, Cm(a.CC, m), Um(a.F, m), a.partmax + (size_t)(m + 1) * G);
            if (!visc_bar()) return false;
            lap<EX>(um, Cm(a.LU, m), Um(a.F, m));
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
                    t1.add((const CT*)Cm(a.LU, m), -dtm * nu_old);
                    Terms t2 = t1;
                    if (m > 0) t1.add((const CT*)C(a.dC), dtm);          // c(u^k_{m-1}) - c(u^{k-1}_{m-1})
                    if (!solve(um, um, t1, dtm * nu_new, Cm(a.LU, m))) return false;
                    if (a.stages == 2) {
                        conv<EX>(um, CONV_OUT, C(a.tmpc), nullptr, nullptr);
                        t2.add((const CT*)C(a.tmpc), dtm);               // c(u^(1))
                        t2.add((const CT*)Cm(a.CC, m), -dtm);            // c(u^{k-1}_m)
                        if (!solve(um, um, t2, dtm * nu_new)) return false;
                    }
                }
                conv<EX>(um, CONV_DELTA, Cm(a.CC, m), Um(a.F, m), a.partmax + (size_t)(m + 1) * G);
                if (!visc_bar()) return false;
                lap<EX>(um, Cm(a.LU, m), Um(a.F, m));
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
        if (a.log_count && blockIdx.x == 0 && threadIdx.x == 0) *a.log_count = log_base + log_n;
        if (blockIdx.x == 0) {
            for (int t = threadIdx.x; t <= MMAX; t += blockDim.x) {
                a.lam[t] = slam_old[t];
                a.lam[MMAX + 1 + t] = slam_new[t];
            }
        }
    }
};

template <int NQ, int DIM, int PDE, bool MIX>
__global__ void __launch_bounds__(512, 1) k_sweep(const __grid_constant__ SweepArgs a) {
    Sweeper<NQ, DIM, PDE, MIX> s(a);
    bool ok;
    if (a.mode == SW_FEVAL) {
        s.feval();
    } else {
        if (a.mode == SW_REFRESH) ok = s.refresh();
        else if (a.mode == SW_PREDICT) ok = s.predict();
        else ok = s.correct();
        if (ok) s.finish();
    }
    grid_exit(a.bar_count, a.bar_exit);
}

template <int NQ, int DIM, int PDE, bool MIX>
size_t sweep_smem(int epb) {
    return Sweeper<NQ, DIM, PDE, MIX>::smem_bytes(epb);
}

template <int NQ, int DIM, int PDE, bool MIX>
int sweep_config_impl(const Geo& g, int* epb_out, int* block_out) {
    using S = Sweeper<NQ, DIM, PDE, MIX>;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int maxepb = S::Q >= 512 ? 1 : 512 / S::Q;
    int epb;
    if (*epb_out > 0) {                            // requested tile size (autotuner)
        epb = *epb_out > maxepb ? maxepb : *epb_out;
    } else {
        long long want = (g.nel + nsm - 1) / nsm;  // aim at one tile per SM
        epb = (int)(want < 1 ? 1 : (want > maxepb ? maxepb : want));
        const int minepb = (32 + S::Q - 1) / S::Q; // at least one warp per block
        if (epb < minepb) epb = minepb > maxepb ? maxepb : minepb;
    }
    const int bs = warp_round(epb * S::Q);
    const size_t sh = sweep_smem<NQ, DIM, PDE, MIX>(epb);
    // the attribute covers the largest tile, so that levels of the same degree
    // with other tile sizes stay launchable
    cudaFuncSetAttribute(k_sweep<NQ, DIM, PDE, MIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep_smem<NQ, DIM, PDE, MIX>(maxepb));
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<NQ, DIM, PDE, MIX>, bs, sh) != cudaSuccess ||
        per < 1)
        return 0;
    const long long ntiles = (g.nel + epb - 1) / epb;
    long long grid = (long long)per * nsm;
    if (grid > ntiles) grid = ntiles;
    *epb_out = epb;
    *block_out = bs;
    return (int)grid;
}

template <int NQ, int DIM, int PDE, bool MIX>
cudaError_t sweep_launch_impl(const SweepArgs& a, int grid, int block) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = sweep_smem<NQ, DIM, PDE, MIX>(a.epb);
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep<NQ, DIM, PDE, MIX>, a);
}

}  // namespace sisdc
