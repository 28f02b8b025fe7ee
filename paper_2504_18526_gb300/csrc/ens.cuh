// Persistent cooperative SI-SDC sweep kernel for an ensemble of independent
// 2D convection-diffusion problems of one polynomial degree (sm_103a).
//
// The ensemble's instances differ in element grid, viscosity, velocity and
// time step.  Their elements are concatenated into one level; the level is
// cut into tiles of `epb` elements that never straddle two instances, and the
// persistent blocks take the tiles round-robin (tile t -> block t mod G), so
// every block holds a mix of instances and the work of a CG iteration stays
// balanced even when instances converge after different iteration counts:
// a converged instance's tiles simply drop out.
//
// Each instance runs its own method (Algorithm 1 with the SI(1)/SI(2)
// deltas of Sec. 3.3 and Sec. 4.3) and its own Jacobi-PCG on
// (M + c_i A) x = M b with c_i = dt_{i,m} nu_tilde_i, nu_tilde_i =
// nu_i + dt_{i,m}/2 lam_i^2 (lam_i = max(|a_x|, |a_y|): the PDE is linear, so
// no spectral-radius reduction is needed).  Inner products are per instance
// and deterministic: a block sums its tiles of instance i into one partial
// part[slot][i][block]; every block that needs the total adds the partials
// of the blocks that own tiles of i in a fixed order, so all blocks see the
// same bits.  The loop over CG iterations runs while any instance is active;
// whether any is left is learnt one phase late from per-block counts.
//
// MIX = true: FP32 inner PCG with FP64 iterative refinement per instance
// (the same scheme as the single-problem kernel); explicit operators and all
// caches stay FP64.
#pragma once
#include <type_traits>

#include "ds.cuh"
#include "ops.h"
#include "pde.cuh"
#include "sipg.cuh"

namespace sisdc {

// per-block state of one instance during an implicit solve
struct EnsLocal {
    double c;        // implicit coefficient dt_m nu_tilde
    double rz;       // (inner) CG residual norm r^T D^-1 r
    double tol2;     // stopping threshold rtol^2 b^T D^-1 b
    double beta, alpha;
    double tol_in;   // inner threshold (MIX)
    int it;          // CG iterations (MIX: inner iterations over all refinements)
    int act;         // CG loop active
    int oact;        // refinement loop active (MIX)
    int ir;          // refinement passes (MIX)
    int fin, done;
};

template <int NQ, bool MIX>
struct EnsSweeper {
    using RT = typename std::conditional<MIX, float, double>::type;
    static constexpr int Q = NQ * NQ;
    static constexpr int TRS = 4 * 2 * NQ;
    static constexpr int NSLOT = 4;          // partial-sum slots per set (two sets alternate)
    static constexpr int NCO = 2 * NQ + 8;   // coefficients per node of the pre-scaled operator
    static constexpr int NTAB = NCO * Q + 4 * NQ;

    static size_t smem_bytes(int epb) {
        const size_t d = NTAB + 2 * Q + 2 * NQ * NQ + 2 * NQ + 32 + 2 * 3 * 32 + (size_t)epb * Q +
                         (size_t)epb * TRS + (size_t)epb * 2 * Q;
        const size_t r = MIX ? (NTAB + 2 * NQ * NQ + NQ + (size_t)epb * Q + (size_t)epb * TRS) : 0;
        return ENS_LSMEM * sizeof(EnsInst) + d * sizeof(double) + r * sizeof(RT) + 16;
    }

    const EnsArgs& a;
    EnsInst* sI;          // the block's instances (shared memory): all of them when
                          // nloc <= ENS_LSMEM (pre), else the current tile's in slot 0
    bool pre;
    double *sA, *sDh, *sWW, *sIWW, *sD, *sK, *sw, *sdl, *scratch, *wsum, *su, *sf, *sF;
    RT *rA, *rDh, *rD, *rK, *rw, *ru, *rf;
    int le, node, i, j, G;
    int solve_parity;
    EnsLocal* L;          // this block's per-instance state [nloc]
    double* dinv_tab;     // this block's Jacobi factors [nloc][Q]
    float* dinv32;        // the same rounded to FP32 (mixed form)
    int nloc;
    const int* loc_inst;  // this block's instances [nloc]

    __device__ EnsSweeper(const EnsArgs& args) : a(args) {
        extern __shared__ double sm[];
        sI = reinterpret_cast<EnsInst*>(sm);
        sA = sm + ENS_LSMEM * sizeof(EnsInst) / sizeof(double);   // [NCO][Q] unit-element operator
        sDh = sA + NCO * Q;                                        // [4][NQ] unit-element face rows
        sWW = sDh + 4 * NQ;                                        // [Q] w_i w_j
        sIWW = sWW + Q;                                            // [Q] 1 / (w_i w_j)
        sD = sIWW + Q;
        sK = sD + NQ * NQ;
        sw = sK + NQ * NQ;
        sdl = sw + NQ;
        scratch = sdl + NQ;
        wsum = scratch + 32;      // [2][3][32] per-warp sums of the last two tiles
        su = wsum + 2 * 3 * 32;
        sf = su + a.epb * Q;
        sF = sf + a.epb * TRS;
        RT* rb = reinterpret_cast<RT*>(sF + a.epb * 2 * Q);
        if (MIX) {
            rA = rb;
            rDh = rA + NCO * Q;
            rD = rDh + 4 * NQ;
            rK = rD + NQ * NQ;
            rw = rK + NQ * NQ;
            ru = rw + NQ;
            rf = ru + a.epb * Q;
        } else {
            rA = reinterpret_cast<RT*>(sA);
            rDh = reinterpret_cast<RT*>(sDh);
            rD = reinterpret_cast<RT*>(sD);
            rK = reinterpret_cast<RT*>(sK);
            rw = reinterpret_cast<RT*>(sw);
            ru = reinterpret_cast<RT*>(su);
            rf = reinterpret_cast<RT*>(sf);
        }
        for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
            sD[t] = a.D[t];
            sK[t] = a.K[t];
            if (MIX) {
                rD[t] = (RT)a.D[t];
                rK[t] = (RT)a.K[t];
            }
        }
        for (int t = threadIdx.x; t < NQ; t += blockDim.x) {
            sw[t] = a.w[t];
            sdl[t] = a.dl[t];
            if (MIX) rw[t] = (RT)a.w[t];
        }
        {
            const UnitElementGeo ug(NQ);
            for (int t = threadIdx.x; t < NCO * Q; t += blockDim.x) {
                const int k = t / Q, nd = t - k * Q;
                const double v = sipg_opA_coeff<NQ, 2>(ug, a.D, a.K, a.w, k, nd % NQ, nd / NQ);
                sA[t] = v;
                if (MIX) rA[t] = (RT)v;
            }
            for (int t = threadIdx.x; t < 4 * NQ; t += blockDim.x) {
                const int f = t / NQ, q = t - f * NQ;
                const double v = 0.5 * a.D[((f & 1) ? NQ - 1 : 0) * NQ + q];
                sDh[t] = v;
                if (MIX) rDh[t] = (RT)v;
            }
            for (int t = threadIdx.x; t < Q; t += blockDim.x) {
                sWW[t] = a.w[t % NQ] * a.w[t / NQ];
                sIWW[t] = 1.0 / sWW[t];
            }
        }
        le = threadIdx.x / Q;
        node = threadIdx.x - le * Q;
        i = node % NQ;
        j = node / NQ;
        G = gridDim.x;
        solve_parity = 0;
        nloc = a.nloc[blockIdx.x];
        loc_inst = a.loc_inst + (size_t)blockIdx.x * a.lmax;
        L = reinterpret_cast<EnsLocal*>(a.loc) + (size_t)blockIdx.x * a.lmax;
        dinv_tab = a.loc_dinv + (size_t)blockIdx.x * a.lmax * Q;
        dinv32 = a.loc_dinv32 + (size_t)blockIdx.x * a.lmax * Q;
        pre = nloc <= ENS_LSMEM;
        if (pre) {
            const int words = (int)(sizeof(EnsInst) / 8);
            for (int t = threadIdx.x; t < nloc * words; t += blockDim.x) {
                const int li = t / words, k = t - li * words;
                reinterpret_cast<unsigned long long*>(sI + li)[k] =
                    __ldg(reinterpret_cast<const unsigned long long*>(a.inst + loc_inst[li]) + k);
            }
        }
        __syncthreads();
    }

    // ---- instance geometry --------------------------------------------------------
    // local instance li (global index inst): from the preloaded table, or
    // staged into slot 0 (block-wide; contains barriers)
    __device__ const EnsInst& inst_of(int li, int inst) {
        if (pre) return sI[li];
        return load_inst(inst);
    }
    __device__ const EnsInst& load_inst(int inst) {
        __syncthreads();
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.inst + inst);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(sI);
        for (int t = threadIdx.x; t < (int)(sizeof(EnsInst) / 8); t += blockDim.x) dst[t] = __ldg(src + t);
        __syncthreads();
        return *sI;
    }

    __device__ void mass_diag(const EnsInst& I, int ii, int jj, double& ms, double& dg) const {
        const double mx = 0.5 * I.hx * sw[ii], my = 0.5 * I.hy * sw[jj];
        ms = mx * my;
        dg = my * (sdl[ii] * I.ihx) + mx * (sdl[jj] * I.ihy);
    }

    __device__ static double nut(const EnsInst& I, double dtm) { return I.nu + 0.5 * dtm * I.lam * I.lam; }

    __device__ long long neighbour(const EnsInst& I, long long e, int f) const {
        const int el = (int)(e - I.e0), ey = el / I.nex, ex = el - ey * I.nex;   // instances hold < 2^31 elements
        int n;
        if (f == 0) n = el + (ex == 0 ? I.nex - 1 : -1);
        else if (f == 1) n = el + (ex == I.nex - 1 ? 1 - I.nex : 1);
        else if (f == 2) n = ey == 0 ? el + (I.ney - 1) * I.nex : el - I.nex;
        else n = ey == I.ney - 1 ? ex : el + I.nex;
        return I.e0 + n;
    }

    // mass of the thread's node in instance I (diagonal GLL mass)
    __device__ double mass_of(const EnsInst& I) const { return I.mq * sWW[node]; }

    __device__ static int line_node(int f, int k, int q) { return f < 2 ? k * NQ + q : q * NQ + k; }

    __device__ bool bar() { return grid_barrier(a.bar_count, a.bar_exit, a.err); }

    // Loop over the block's tiles: fn(I, e0, nle, li, acc[K]) accumulates K
    // per-thread values; their block sums go to part[slot0 + k][inst][block].
    // Tiles of instances whose EnsLocal::act (or oact) is 0 are skipped when
    // `which` is 1 (or 2).
    template <int K, class Fn>
    __device__ void tiles(double* part, int which, Fn fn) {
        // thread 0 keeps the running sums of the current instance (cur); the
        // warp sums of a tile are added after the tile's closing barrier, in
        // warp order, so every sum has a fixed order
        double run[K > 0 ? K : 1];
        int cur = -1, pend = -1, pbuf = 0, buf = 0;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < K; ++k) run[k] = 0.0;
        auto consume = [&]() {
            if (cur != pend) {
                if (cur >= 0)
                    for (int k = 0; k < K; ++k) part[((size_t)k * a.ninst + cur) * G + blockIdx.x] = run[k];
                cur = pend;
                for (int k = 0; k < K; ++k) run[k] = 0.0;
            }
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += wsum[(pbuf * 3 + k) * 32 + w];
                run[k] += s;
            }
        };
        for (long long t = blockIdx.x; t < a.ntiles; t += G) {
            const int4 td = __ldg(a.tiles + t);       // (instance, local index, first element, elements)
            if (which == 1 && !L[td.y].act) continue;
            if (which == 2 && !L[td.y].oact) continue;
            if (K > 0 && threadIdx.x == 0 && pend >= 0) consume();
            const EnsInst& I = inst_of(td.y, td.x);
            double acc[K > 0 ? K : 1];
            for (int k = 0; k < K; ++k) acc[k] = 0.0;
            fn(I, (long long)td.z, td.w, td.y, acc);
            if (K > 0) {
                for (int k = 0; k < K; ++k) {
                    const double v = warp_sum(acc[k]);
                    if (lane == 0) wsum[(buf * 3 + k) * 32 + wid] = v;
                }
                pend = td.x;
                pbuf = buf;
                buf ^= 1;
            }
            __syncthreads();
        }
        if (K > 0 && threadIdx.x == 0) {
            if (pend >= 0) consume();
            if (cur >= 0)
                for (int k = 0; k < K; ++k) part[((size_t)k * a.ninst + cur) * G + blockIdx.x] = run[k];
        }
    }

    // total of slot k of instance loc_inst[li] for every local instance that
    // passes `sel`; store(li, total) runs on one lane per instance
    template <class Sel, class Store>
    __device__ void totals(const double* part, int k, Sel sel, Store store) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = max(1, (int)(blockDim.x >> 5));
        for (int li = w; li < nloc; li += nw) {
            if (!sel(L[li])) continue;
            const int inst = loc_inst[li];
            const int t0 = __ldg(&a.inst[inst].t0);
            const int nt = __ldg(&a.inst[inst].nt);
            const int n = nt < G ? nt : G;
            const double* p = part + ((size_t)k * a.ninst + inst) * G;
            double v = 0.0;
            for (int q = lane; q < n; q += 32) v += __ldcg(p + (t0 + q) % G);
            v = warp_sum(v);
            if (lane == 0) store(L[li], v);
        }
        __syncthreads();
    }

    // number of this block's instances with the given flag set -> cnt[block]
    __device__ void count_active(double* cnt, int which) {
        if (threadIdx.x == 0) {
            int n = 0;
            for (int li = 0; li < nloc; ++li) n += which == 1 ? L[li].act : L[li].oact;
            cnt[blockIdx.x] = (double)n;
        }
    }
    __device__ double grid_sum(const double* cnt) { return grid_total(cnt, scratch); }

    // ---- SIPG faces of a tile ----------------------------------------------------
    template <class V, class GetV>
    __device__ void faces(const EnsInst& I, int nle, long long e0, const V* tu, V* tf, const V* Dh, GetV getv) {
        const int per = 4 * NQ;
        for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
            const int l = t / per;
            const int rem = t - l * per;
            const int f = rem / NQ, k = rem - f * NQ;
            const long long en = neighbour(I, e0 + l, f);
            const V* u = tu + l * Q;
            V vo[NQ], vn[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                vo[q] = u[line_node(f, k, q)];
                vn[q] = getv(en, line_node(f ^ 1, k, q));
            }
            V jump, avg;     // avg: the unscaled derivative average of the unit element
            sipg_face_pre<NQ>(vo, vn, f, Dh, jump, avg);
            V* o = tf + (l * 4 + f) * 2 * NQ;
            o[k] = jump;
            o[NQ + k] = avg;
        }
    }

    // Face traces of a tile's elements from their nodal values in shared memory:
    // per face f and row k the value at the face node and the half-scaled
    // normal derivative sum_q Dh[f][q] u(line) -- the two numbers a neighbour
    // needs to form the SIPG jump and average across that face.
    __device__ void write_traces(int nle, long long e0, const double* tu, double* T) const {
        const int per = 4 * NQ;
        for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
            const int l = t / per, rem = t - l * per, f = rem / NQ, k = rem - f * NQ;
            const double* u = tu + l * Q;
            const double* ro = sDh + f * NQ;
            double d = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) d += ro[q] * u[line_node(f, k, q)];
            double* o = T + ((e0 + l) * 4 + f) * 2 * NQ;
            o[k] = u[line_node(f, k, (f & 1) ? NQ - 1 : 0)];
            o[NQ + k] = d;
        }
    }

    // SIPG face data of the new search direction p = z + beta p_old from the
    // traces of z and p_old (the traces are linear in the nodal values): own
    // faces also store p's traces for the next iteration
    __device__ void faces_traced(const EnsInst& I, int nle, long long e0, double beta, const double* Tpold,
                                 double* Tpcur) {
        const int per = 4 * NQ;
        for (int t = threadIdx.x; t < nle * per; t += blockDim.x) {
            const int l = t / per, rem = t - l * per, f = rem / NQ, k = rem - f * NQ;
            const long long e = e0 + l, en = neighbour(I, e, f);
            const long long oo = (e * 4 + f) * 2 * NQ + k, on = (en * 4 + (f ^ 1)) * 2 * NQ + k;
            double vo = __ldcg(a.tz + oo), dd = __ldcg(a.tz + oo + NQ);
            double vn = __ldcg(a.tz + on), dn = __ldcg(a.tz + on + NQ);
            if (beta != 0.0) {
                vo += beta * __ldcg(Tpold + oo);
                dd += beta * __ldcg(Tpold + oo + NQ);
                vn += beta * __ldcg(Tpold + on);
                dn += beta * __ldcg(Tpold + on + NQ);
            }
            Tpcur[oo] = vo;
            Tpcur[oo + NQ] = dd;
            double* o = sf + (l * 4 + f) * 2 * NQ;
            o[k] = (f & 1) ? vo - vn : vn - vo;
            o[NQ + k] = dd + dn;
        }
    }

    // (A u) of the thread's node: unit-element sums scaled by the instance's aspect ratio
    template <class V>
    __device__ V opA(const EnsInst& I, const V* tu, const V* tf, const V* cf) const {
        V X, Y;
        sipg_opA_pre_xy<NQ>(i, j, tu + le * Q, tf + le * TRS, cf + node, X, Y);
        return V(I.rho) * X + V(I.irho) * Y;
    }

    __device__ static double znew(double z, double beta, double pold) { return beta == 0.0 ? z : z + beta * pold; }

    template <class V>
    __device__ static V pnew(V r, V dinv, V beta, V pold) {
        const V z = r * dinv;
        return beta == V(0) ? z : z + beta * pold;
    }

    // right-hand side b = u_prev + Q_m + G_m - dt_m nu_tilde L u_m + fa dt_m A + fb dt_m B
    struct Rhs {
        const double *up, *Qm, *Gm, *LUm, *A, *B;
        double fa, fb;
    };
    __device__ static double rhs_at(const Rhs& R, long long id, double dtm, double nt) {
        double b = __ldcg(R.up + id);
        if (R.Qm) b += __ldcg(R.Qm + id);
        if (R.Gm) b += __ldcg(R.Gm + id);
        if (R.LUm) b += (-dtm * nt) * __ldcg(R.LUm + id);
        if (R.A) b += (R.fa * dtm) * __ldcg(R.A + id);
        if (R.B) b += (R.fb * dtm) * __ldcg(R.B + id);
        return b;
    }

    // per-instance implicit coefficient and Jacobi factors of node m
    __device__ void set_coeffs(int m) {
        if (pre) {
            __syncthreads();
            for (int t = threadIdx.x; t < nloc * Q; t += blockDim.x) {
                const int li = t / Q, q = t - li * Q;
                const EnsInst& I = sI[li];
                const double dtm = I.dt * a.dtau[m];
                const double c = dtm * nut(I, dtm);
                double ms, dg;
                mass_diag(I, q % NQ, q / NQ, ms, dg);
                const double dv = 1.0 / (ms + c * dg);
                dinv_tab[(size_t)li * Q + q] = dv;
                if (MIX) dinv32[(size_t)li * Q + q] = d2f_int(dv);
            }
        }
        for (int li = 0; li < nloc; ++li) {
            const EnsInst& I = pre ? sI[li] : load_inst(loc_inst[li]);
            const double dtm = I.dt * a.dtau[m];
            const double c = dtm * nut(I, dtm);
            if (!pre)
                for (int t = threadIdx.x; t < Q; t += blockDim.x) {
                    double ms, dg;
                    mass_diag(I, t % NQ, t / NQ, ms, dg);
                    const double dv = 1.0 / (ms + c * dg);
                    dinv_tab[(size_t)li * Q + t] = dv;
                    if (MIX) dinv32[(size_t)li * Q + t] = d2f_int(dv);
                }
            if (threadIdx.x == 0) {
                EnsLocal& s = L[li];
                s.c = c;
                s.it = 0;
                s.ir = 0;
                s.beta = 0.0;
                s.act = 1;
                s.oact = 1;
                s.fin = 1;
                s.done = 0;
            }
        }
        __syncthreads();
    }

    // statistics of the finished solve, once per instance (by the owner of its first tile)
    __device__ void stat_solves() {
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int li = 0; li < nloc; ++li) {
                const int inst = loc_inst[li];
                if (__ldg(&a.inst[inst].t0) % G != (int)blockIdx.x) continue;
                const EnsLocal& s = L[li];
                atomicAdd((unsigned long long*)&a.stats[ST_SOLVES], 1ull);
                atomicAdd((unsigned long long*)&a.stats[ST_ITERS], (unsigned long long)s.it);
                atomicMax((unsigned long long*)&a.stats[ST_MAXIT], (unsigned long long)s.it);
                if (MIX) atomicAdd((unsigned long long*)&a.stats[ST_IR], (unsigned long long)(s.ir + 1));
                if (a.inst_iters) a.inst_iters[inst] += s.it;
                if (!s.fin) {
                    atomicOr(a.err, DEV_NONFINITE);
                } else if (!s.done) {
                    atomicOr(a.err, DEV_NOCONV);
                    atomicAdd((unsigned long long*)&a.stats[ST_NOCONV], 1ull);
                }
            }
        }
        __syncthreads();
    }

    // ---- implicit solves of node m: (M + c_i A) x = M b for every instance -------
    // initial guess xsrc (x itself when xsrc == x); Lx0 (nullable) = cached L xsrc
    __device__ bool solve(int m, double* x, const double* xsrc, const Rhs& R, const double* Lx0) {
        double* part = a.part + (size_t)(solve_parity ? NSLOT : 0) * a.ninst * G;
        double* cnt = a.part + (size_t)2 * NSLOT * a.ninst * G;
        solve_parity ^= 1;
        set_coeffs(m);
        if (MIX) return solve_mix(m, x, xsrc, R, Lx0, part, cnt);
        const double rtol2 = a.rtol * a.rtol;
        double* Z = static_cast<double*>(a.rf);    // z = D^-1 r, stored with r
        // initial residual r = M b - (M + c A) x0
        tiles<2>(part, 0, [&](const EnsInst& I, long long e0, int nle, int li, double* acc) {
            const bool act = le < nle;
            const long long e = e0 + le, id = e * Q + node;
            const double c = L[li].c, dinv = dinv_tab[(size_t)li * Q + node];
            if (act) {
                const double xv = __ldcg(xsrc + id);
                su[le * Q + node] = xv;
                if (xsrc != x) x[id] = xv;
            }
            __syncthreads();
            if (!Lx0) faces<double>(I, nle, e0, su, sf, sDh, [&](long long en, int nd) { return __ldcg(xsrc + en * Q + nd); });
            __syncthreads();
            if (act) {
                const double ms = mass_of(I);
                const double dtm = I.dt * a.dtau[m];
                const double mb = ms * rhs_at(R, id, dtm, nut(I, dtm));
                const double xv = su[le * Q + node];
                const double Ax = Lx0 ? -ms * __ldcg(Lx0 + id) : opA<double>(I, su, sf, sA);
                const double rr = mb - (ms * xv + c * Ax);
                const double zz = rr * dinv;
                a.r[id] = rr;
                Z[id] = zz;
                acc[0] += mb * mb * dinv;
                acc[1] += rr * zz;
            }
            if (a.tz) {                                   // traces of z for the first direction
                __syncthreads();
                if (act) su[le * Q + node] = Z[id];
                __syncthreads();
                write_traces(nle, e0, su, a.tz);
            }
        });
        if (!bar()) return false;
        totals(part, 0, [](const EnsLocal&) { return true; }, [&](EnsLocal& s, double v) { s.tol2 = fmax(rtol2 * v, 1e-300); s.fin = isfinite(v); });
        totals(part, 1, [](const EnsLocal&) { return true; }, [&](EnsLocal& s, double v) {
            s.rz = v;
            s.fin = s.fin && isfinite(v);
            s.act = s.fin && v > s.tol2 && a.maxit > 0;
            s.done = s.fin && !(v > s.tol2);
        });
        double* P0 = static_cast<double*>(a.p);
        double* P1 = static_cast<double*>(a.p2);
        double* AP = static_cast<double*>(a.Ap);
        for (int par = 0;; par ^= 1) {
            const double* pold = par ? P1 : P0;
            double* pcur = par ? P0 : P1;
            const double* Tpold = par ? a.tp1 : a.tp0;
            double* Tpcur = par ? a.tp0 : a.tp1;
            count_active(cnt, 1);
            tiles<1>(part + (size_t)2 * a.ninst * G, 1, [&](const EnsInst& I, long long e0, int nle, int li, double* acc) {
                const bool act = le < nle;
                const long long e = e0 + le, id = e * Q + node;
                const double beta = L[li].beta, c = L[li].c;
                double pn = 0.0;
                if (act) {
                    pn = znew(__ldcg(Z + id), beta, beta == 0.0 ? 0.0 : __ldcg(pold + id));
                    pcur[id] = pn;
                    su[le * Q + node] = pn;
                }
                __syncthreads();
                if (a.tz)
                    faces_traced(I, nle, e0, beta, Tpold, Tpcur);
                else
                    faces<double>(I, nle, e0, su, sf, sDh, [&](long long en, int nd) {
                        const long long idn = en * Q + nd;
                        return znew(__ldcg(Z + idn), beta, beta == 0.0 ? 0.0 : __ldcg(pold + idn));
                    });
                __syncthreads();
                if (act) {
                    const double Apv = mass_of(I) * pn + c * opA<double>(I, su, sf, sA);
                    AP[id] = Apv;
                    acc[0] += pn * Apv;
                }
            });
            if (!bar()) return false;
            if (grid_sum(cnt) == 0.0) break;
            totals(part + (size_t)2 * a.ninst * G, 0, [](const EnsLocal& s) { return s.act != 0; },
                   [](EnsLocal& s, double v) { s.alpha = s.rz / v; });
            tiles<1>(part + (size_t)3 * a.ninst * G, 1, [&](const EnsInst&, long long e0, int nle, int li, double* acc) {
                double zz = 0.0;
                if (le < nle) {
                    const long long id = (e0 + le) * Q + node;
                    const double alpha = L[li].alpha, dinv = dinv_tab[(size_t)li * Q + node];
                    x[id] = __ldcg(x + id) + alpha * __ldcg(pcur + id);
                    const double rr = __ldcg(a.r + id) - alpha * __ldcg(AP + id);
                    zz = rr * dinv;
                    a.r[id] = rr;
                    Z[id] = zz;
                    acc[0] += rr * zz;
                }
                if (a.tz) {                               // traces of the new z
                    if (le < nle) su[le * Q + node] = zz;
                    __syncthreads();
                    write_traces(nle, e0, su, a.tz);
                }
            });
            if (!bar()) return false;
            totals(part + (size_t)3 * a.ninst * G, 0, [](const EnsLocal& s) { return s.act != 0; },
                   [&](EnsLocal& s, double v) {
                       s.beta = v / s.rz;
                       s.rz = v;
                       ++s.it;
                       s.fin = isfinite(v);
                       s.done = s.fin && !(v > s.tol2);
                       s.act = s.fin && v > s.tol2 && s.it < a.maxit;
                   });
        }
        stat_solves();
        return true;
    }

    // mixed precision: FP64 refinement residual, FP32 inner PCG, per instance
    __device__ bool solve_mix(int m, double* x, const double* xsrc, const Rhs& R, const double* Lx0, double* part,
                              double* cnt) {
        const double rtol2 = a.rtol * a.rtol;
        RT* RF = static_cast<RT*>(a.rf);
        RT* P0 = static_cast<RT*>(a.p);
        RT* P1 = static_cast<RT*>(a.p2);
        RT* AP = static_cast<RT*>(a.Ap);
        const int max_ir = 30;
        for (int ir = 0; ir < max_ir; ++ir) {
            const double* xs = ir == 0 ? xsrc : x;
            count_active(cnt, 2);
            tiles<3>(part, 2, [&](const EnsInst& I, long long e0, int nle, int li, double* acc) {
                const bool act = le < nle;
                const long long id = (e0 + le) * Q + node;
                const double c = L[li].c, dinv = dinv_tab[(size_t)li * Q + node];
                const RT dinvr = to_v<RT>(dinv);
                if (act) {
                    const double xv = __ldcg(xs + id);
                    su[le * Q + node] = xv;
                    if (ir == 0 && xsrc != x) x[id] = xv;
                }
                __syncthreads();
                if (!(ir == 0 && Lx0))
                    faces<double>(I, nle, e0, su, sf, sDh, [&](long long en, int nd) { return __ldcg(xs + en * Q + nd); });
                __syncthreads();
                if (act) {
                    const double ms = mass_of(I);
                    double mb;
                    if (ir == 0) {
                        const double dtm = I.dt * a.dtau[m];
                        mb = ms * rhs_at(R, id, dtm, nut(I, dtm));
                        a.r[id] = mb;
                        acc[0] += mb * mb * dinv;
                    } else {
                        mb = __ldcg(a.r + id);
                    }
                    const double xv = su[le * Q + node];
                    const double Ax = (ir == 0 && Lx0) ? -ms * __ldcg(Lx0 + id) : opA<double>(I, su, sf, sA);
                    const double r64 = mb - (ms * xv + c * Ax);
                    acc[1] += r64 * (r64 * dinv);
                    const RT r32 = to_v<RT>(r64);
                    RF[id] = r32;
                    acc[2] += to_f64(r32 * (r32 * dinvr));   // FP32 term, FP64 sum
                }
            });
            if (!bar()) return false;
            if (grid_sum(cnt) == 0.0) break;
            if (ir == 0)
                totals(part, 0, [](const EnsLocal&) { return true; }, [&](EnsLocal& s, double v) {
                    s.tol2 = fmax(rtol2 * v, 1e-300);
                    s.fin = isfinite(v);
                });
            // refinement residual: finished, or start an inner solve
            totals(part, 1, [](const EnsLocal& s) { return s.oact != 0; }, [&](EnsLocal& s, double v) {
                s.fin = s.fin && isfinite(v);
                s.ir = ir;
                if (!s.fin || !(v > s.tol2)) {
                    s.done = s.fin;
                    s.oact = 0;
                    s.act = 0;
                }
            });
            totals(part, 2, [](const EnsLocal& s) { return s.oact != 0; }, [&](EnsLocal& s, double v) {
                s.rz = v;
                s.fin = s.fin && isfinite(v);
                s.tol_in = fmax(1e-10 * v, 0.25 * s.tol2);
                s.beta = 0.0;
                s.act = s.oact && s.fin && v > s.tol_in && s.it < a.maxit;
                if (!s.fin) s.oact = 0;
            });
            for (int par = 0;; par ^= 1) {
                const RT* pold = par ? P1 : P0;
                RT* pcur = par ? P0 : P1;
                count_active(cnt + G, 1);
                tiles<1>(part + (size_t)3 * a.ninst * G, 1, [&](const EnsInst& I, long long e0, int nle, int li, double* acc) {
                    const bool act = le < nle;
                    const long long id = (e0 + le) * Q + node;
                    const RT betar = (RT)L[li].beta, cr = (RT)L[li].c;
                    const float* dv = dinv32 + (size_t)li * Q;
                    RT pn = RT(0);
                    if (act) {
                        pn = pnew<RT>(__ldcg(RF + id), RT(dv[node]), betar, betar == RT(0) ? RT(0) : __ldcg(pold + id));
                        pcur[id] = pn;
                        ru[le * Q + node] = pn;
                    }
                    __syncthreads();
                    faces<RT>(I, nle, e0, ru, rf, rDh, [&](long long en, int nd) {
                        const long long idn = en * Q + nd;
                        return pnew<RT>(__ldcg(RF + idn), RT(dv[nd]), betar, betar == RT(0) ? RT(0) : __ldcg(pold + idn));
                    });
                    __syncthreads();
                    if (act) {
                        const RT Apv = to_v<RT>(mass_of(I)) * pn + cr * opA<RT>(I, ru, rf, rA);
                        AP[id] = Apv;
                        acc[0] += to_f64(pn * Apv);
                    }
                });
                if (!bar()) return false;
                if (grid_sum(cnt + G) == 0.0) break;
                totals(part + (size_t)3 * a.ninst * G, 0, [](const EnsLocal& s) { return s.act != 0; },
                       [](EnsLocal& s, double v) { s.alpha = s.rz / v; });
                // the slot of the refinement's M b norm is free again: reuse slot 0
                tiles<1>(part, 1, [&](const EnsInst&, long long e0, int nle, int li, double* acc) {
                    if (le < nle) {
                        const long long id = (e0 + le) * Q + node;
                        const double alpha = L[li].alpha;
                        const RT alphar = (RT)alpha, dinvr = RT(dinv32[(size_t)li * Q + node]);
                        x[id] = __ldcg(x + id) + alpha * to_f64(__ldcg(pcur + id));
                        const RT rr = __ldcg(RF + id) - alphar * __ldcg(AP + id);
                        RF[id] = rr;
                        acc[0] += to_f64(rr * (rr * dinvr));
                    }
                });
                if (!bar()) return false;
                totals(part, 0, [](const EnsLocal& s) { return s.act != 0; }, [&](EnsLocal& s, double v) {
                    s.beta = v / s.rz;
                    s.rz = v;
                    ++s.it;
                    const bool f = isfinite(v);
                    s.act = f && v > s.tol_in && s.it < a.maxit;
                    if (s.it >= a.maxit) s.oact = 0;
                });
            }
        }
        stat_solves();
        return true;
    }

    // ---- explicit operators ------------------------------------------------------
    // c(X) into out; CONV_DELTA also writes dC = c - out_old; f64 (optional)
    // receives c (the start of the cached f)
    // One face node of c(u) (local element l, side 0/1 of direction x (XD)
    // or y, face row k): the lifted Rusanov-minus-own flux difference, the
    // correction of c(u) at the own end node, into the face buffer [l][f][k]
    template <bool XD>
    __device__ void conv_face(const EnsInst& I, const PdeParams& pp, const double* X, long long e0, int l, int side,
                              int k) const {
        const int f = (XD ? 0 : 2) + side;
        const int io = side ? NQ - 1 : 0, in = NQ - 1 - io;
        const int nd = XD ? k * NQ + io : io * NQ + k;
        const int ndn = XD ? k * NQ + in : in * NQ + k;
        const long long e = e0 + l;
        const double uo = __ldcg(X + e * Q + nd);
        const double un = __ldcg(X + neighbour(I, e, f) * Q + ndn);
        double d;
        rusanov_jump<0, XD>(pp, &uo, &un, side == 1, &d);
        const double lift = XD ? (side ? -I.liftRx : I.liftLx) : (side ? -I.liftRy : I.liftLy);
        sf[(size_t)l * TRS + f * NQ + k] = lift * d;
    }

    __device__ void conv(const double* X, int mode, double* out, double* f64) {
        tiles<0>(nullptr, 0, [&](const EnsInst& I, long long e0, int nle, int, double*) {
            const bool act = le < nle;
            const long long e = e0 + le, id = e * Q + node;
            const PdeParams pp{0.0, I.ax, I.ay};
            double* sFx = sF + (size_t)le * 2 * Q;
            double* sFy = sFx + Q;
            if (act) {
                const double u = __ldcg(X + id);
                double Fx, Fy;
                Pde<0>::fx(pp, &u, &Fx);
                Pde<0>::fy(pp, &u, &Fy);
                sFx[node] = Fx;
                sFy[node] = Fy;
            }
            // face tasks, one per face node: x faces, then y faces from the next whole warp
            {
                const int nx = nle * 2 * NQ, xr = (nx + 31) & ~31;
                for (int t = threadIdx.x; t < xr + nx; t += blockDim.x) {
                    if (t < nx) {
                        const int l = t / (2 * NQ), r = t - l * 2 * NQ;
                        conv_face<true>(I, pp, X, e0, l, r / NQ, r % NQ);
                    } else if (t >= xr) {
                        const int ty = t - xr, l = ty / (2 * NQ), r = ty - l * 2 * NQ;
                        conv_face<false>(I, pp, X, e0, l, r / NQ, r % NQ);
                    }
                }
            }
            __syncthreads();
            if (act) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < NQ; ++k) s += sD[i * NQ + k] * sFx[j * NQ + k];
                double cv = -I.sx * s;
                s = 0.0;
#pragma unroll
                for (int k = 0; k < NQ; ++k) s += sD[j * NQ + k] * sFy[k * NQ + i];
                cv -= I.sy * s;
                const double* fc = sf + (size_t)le * TRS;
                if (i == 0) cv += fc[j];
                if (i == NQ - 1) cv += fc[NQ + j];
                if (j == 0) cv += fc[2 * NQ + i];
                if (j == NQ - 1) cv += fc[3 * NQ + i];
                if (mode == CONV_DELTA) a.dC[id] = cv - __ldcg(out + id);
                out[id] = cv;
                if (f64) f64[id] = cv;
            }
        });
    }

    // LU = L X; F += nu LU, F holding c(X) from the conv phase of the same block
    __device__ void lap(const double* X, double* LUm, double* Fm) {
        tiles<0>(nullptr, 0, [&](const EnsInst& I, long long e0, int nle, int, double*) {
            const bool act = le < nle;
            const long long id = (e0 + le) * Q + node;
            if (act) su[le * Q + node] = __ldcg(X + id);
            __syncthreads();
            faces<double>(I, nle, e0, su, sf, sDh, [&](long long en, int nd) { return __ldcg(X + en * Q + nd); });
            __syncthreads();
            if (act) {
                const double lu = -opA<double>(I, su, sf, sA) * (I.imq * sIWW[node]);
                LUm[id] = lu;
                Fm[id] = __ldcg(Fm + id) + I.nu * lu;
            }
        });
    }

    // out = u_prev + Q_m + G_m (Lobatto first node)
    __device__ void copy_node(double* out, const double* up, const double* Qm, const double* Gm) {
        tiles<0>(nullptr, 0, [&](const EnsInst&, long long e0, int nle, int, double*) {
            if (le < nle) {
                const long long id = (e0 + le) * Q + node;
                double v = __ldcg(up + id);
                if (Qm) v += __ldcg(Qm + id);
                if (Gm) v += __ldcg(Gm + id);
                out[id] = v;
            }
        });
    }

    // Q_m = dt_i sum_j W[m][j] F_j (FP64 accumulation)
    __device__ void quad() {
        const long long N = a.N;
        tiles<0>(nullptr, 0, [&](const EnsInst& I, long long e0, int nle, int, double*) {
            if (le < nle) {
                const long long id = (e0 + le) * Q + node;
                double f[MMAX];
#pragma unroll
                for (int q = 0; q < MMAX; ++q) f[q] = q < a.M ? __ldcg(a.F + q * N + id) : 0.0;
#pragma unroll
                for (int mm = 0; mm < MMAX; ++mm) {
                    if (mm >= a.M) break;
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < MMAX; ++q)
                        if (q < a.M) s += a.W[mm * a.M + q] * f[q];
                    a.Qb[mm * N + id] = I.dt * s;
                }
            }
        });
    }

    __device__ double* Um(double* U, int m) const { return U + (long long)m * a.N; }
    __device__ const double* Um(const double* U, int m) const { return U + (long long)m * a.N; }

    // ---- the three modes ---------------------------------------------------------
    __device__ bool refresh() {
        conv(a.u0, CONV_OUT, a.c0, nullptr);
        for (int m = 0; m < a.M; ++m) {
            conv(Um(a.U, m), CONV_OUT, Um(a.CC, m), Um(a.F, m));
            lap(Um(a.U, m), Um(a.LU, m), Um(a.F, m));
        }
        return true;
    }

    __device__ bool predict() {
        conv(a.u0, CONV_OUT, a.c0, nullptr);
        if (!bar()) return false;
        for (int m = 0; m < a.M; ++m) {
            const double* up = m ? Um((const double*)a.U, m - 1) : a.u0;
            const double* cp = m ? Um((const double*)a.CC, m - 1) : a.c0;
            double* um = Um(a.U, m);
            if (a.dtau[m] != 0.0) {
                Rhs r1{up, nullptr, nullptr, nullptr, cp, nullptr, 1.0, 0.0};
                if (!solve(m, um, up, r1, m ? Um((const double*)a.LU, m - 1) : nullptr)) return false;
                if (a.stages == 2) {
                    conv(um, CONV_OUT, a.tmpc, nullptr);
                    Rhs r2{up, nullptr, nullptr, nullptr, a.tmpc, nullptr, 1.0, 0.0};
                    if (!solve(m, um, um, r2, nullptr)) return false;
                }
            } else {
                copy_node(um, up, nullptr, nullptr);
                if (!bar()) return false;
            }
            conv(um, CONV_OUT, Um(a.CC, m), Um(a.F, m));
            lap(um, Um(a.LU, m), Um(a.F, m));
            if (!bar()) return false;
        }
        return true;
    }

    __device__ bool correct() {
        for (int k = 0; k < a.nsweeps; ++k) {
            quad();
            for (int m = 0; m < a.M; ++m) {
                const double* up = m ? Um((const double*)a.U, m - 1) : a.u0;
                double* um = Um(a.U, m);
                const double* Qm = Um((const double*)a.Qb, m);
                const double* Gm = a.G ? Um(a.G, m) : nullptr;
                if (a.dtau[m] == 0.0) {
                    copy_node(um, up, Qm, Gm);
                    if (!bar()) return false;
                } else {
                    Rhs r1{up, Qm, Gm, Um((const double*)a.LU, m), m > 0 ? (const double*)a.dC : nullptr, nullptr, 1.0, 0.0};
                    if (!solve(m, um, um, r1, Um((const double*)a.LU, m))) return false;
                    if (a.stages == 2) {
                        conv(um, CONV_OUT, a.tmpc, nullptr);
                        Rhs r2{up, Qm, Gm, Um((const double*)a.LU, m), a.tmpc, Um((const double*)a.CC, m), 1.0, -1.0};
                        if (!solve(m, um, um, r2, nullptr)) return false;
                    }
                }
                conv(um, CONV_DELTA, Um(a.CC, m), Um(a.F, m));
                lap(um, Um(a.LU, m), Um(a.F, m));
                if (!bar()) return false;
            }
        }
        return true;
    }
};

// MINB = 1: up to 128 registers per thread (one 512-thread block per SM);
// MINB = 2: at most 64 (two such blocks, or four of 256 threads, per SM) --
// more resident warps to hide the FP64 and shared-memory latencies, fewer
// registers per thread.  The same arithmetic per thread; the host picks the
// capped kernel when a level's grid has more blocks than the plain kernel
// keeps resident (the tile-to-block assignment, and with it the order of the
// per-instance partial sums, follows the grid).
template <int NQ, bool MIX, int MINB>
__global__ void __launch_bounds__(512, MINB) k_ens_sweep(const __grid_constant__ EnsArgs a) {
    EnsSweeper<NQ, MIX> s(a);
    if (a.mode == SW_REFRESH) s.refresh();
    else if (a.mode == SW_PREDICT) s.predict();
    else s.correct();
    grid_exit(a.bar_count, a.bar_exit);
}

template <int NQ, bool MIX>
size_t ens_smem(int epb) {
    return EnsSweeper<NQ, MIX>::smem_bytes(epb);
}

// blocks per SM for a block of epb*Q threads (0 if it cannot run)
template <int NQ, bool MIX, int MINB = 1>
int ens_occupancy_impl(int epb) {
    if (epb < 1 || epb * NQ * NQ > 512) return 0;
    const int bs = warp_round(epb * NQ * NQ);
    const size_t sh = ens_smem<NQ, MIX>(epb);
    // the attribute covers the largest tile, so that every shape stays launchable
    const size_t shmax = ens_smem<NQ, MIX>(512 / (NQ * NQ));
    if (cudaFuncSetAttribute(k_ens_sweep<NQ, MIX, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmax) !=
        cudaSuccess)
        return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ens_sweep<NQ, MIX, MINB>, bs, sh) != cudaSuccess)
        return 0;
    return per;
}

template <int NQ, bool MIX, int MINB = 1>
cudaError_t ens_launch_impl(const EnsArgs& a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)warp_round(a.epb * NQ * NQ));
    cfg.dynamicSmemBytes = ens_smem<NQ, MIX>(a.epb);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_ens_sweep<NQ, MIX, MINB>, a);
}

}  // namespace sisdc
