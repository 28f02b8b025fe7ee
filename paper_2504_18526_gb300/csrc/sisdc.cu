// Host orchestration and C ABI of the SI-MLSDC library.
//
// All arithmetic runs in the kernels of ops_*.cu; this file queues them on
// the context stream in the order of the method:
//   sweep     Algorithm 1 with the SI(1)/SI(2) deltas (Sec. 3.3, Sec. 4.3)
//   predictor eqs. sdc:incremental_predictor_si1/_si2
//   vcycle    Algorithm 2 (FAS right-hand side, eq. ml-cm:incremental:fas-mg:rhs)
//   start     Algorithms 3 (Cascade) and 4 (FMG, one cycle per added level)
// The cached f, c and L u of the previous sweep (Sec. 3.3 implementation
// remark) live in per-level device arrays; the nu_tilde factors are read by
// the kernels from device-side spectral-radius slots, so a whole time step
// is queued without a host synchronisation and can be captured as one CUDA
// graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sisdc.h"
#include "ops.h"
#include "tables.h"

using namespace sisdc;

struct sisdc_level_s {
    sisdc_ctx_s* ctx = nullptr;
    int index = 0;
    bool mix = false;            // this level runs the mixed-precision form
    sisdc_level_desc desc{};
    LevelTables tab;
    Geo geo{};
    int nq = 0, nqy = 0, Q = 0, M = 0, nel = 0;
    long long N = 0, NV = 0;
    double* d_tab = nullptr;
    double* d_mem = nullptr;
    size_t tab_bytes = 0, mem_bytes = 0;
    // state and caches
    double *U = nullptr, *u0 = nullptr;
    double *F = nullptr, *CC = nullptr, *LU = nullptr, *Qb = nullptr, *G = nullptr, *V = nullptr, *R = nullptr;
    double *c0 = nullptr, *dC = nullptr, *tmpc = nullptr;
    double *cg_r = nullptr, *cg_p = nullptr, *cg_Ap = nullptr, *trx = nullptr, *trp = nullptr;
    double* cg_p2 = nullptr;    // second search-direction buffer of the sweep kernel
    double* cg_rf = nullptr;    // FP32 inner residual of the mixed-precision refinement; FP64 form: z = D^-1 r
    double* FV = nullptr;       // Navier-Stokes viscous fluxes [6][N]
    int sw_grid = 0, sw_epb = 0, sw_block = 0;
    double* lam = nullptr;      // [2][MMAX+1]: old, new spectral radius slots
    int pcg_grid = 0, pcg_block = 0;
    bool valid = false;         // caches match (u0, U)
    const double* cache_u0 = nullptr;
    const double* cache_U = nullptr;
    // transfers to the next coarser level
    double *d_Ix = nullptr, *d_Px = nullptr, *d_Rx = nullptr;
    double *d_It = nullptr, *d_Pt = nullptr, *d_Rt = nullptr, *d_one = nullptr;
    // element ratio to the next coarser level per direction (1, or 2: 2:1
    // h-coarsening); with a ratio 2 the x tables above hold one matrix per
    // child and the y tables below are used
    int rx = 1, ry = 1;
    double *d_Iy = nullptr, *d_Py = nullptr, *d_Ry = nullptr;
    // learned initial guess of the implicit solves of this level's correction
    // sweeps (sisdc_set_learned); nullptr = the persistent sweep kernel
    sisdc_mlp learned = nullptr;
    // artificial viscosity (sisdc_set_av): modal matrix, per-element
    // viscosities [M][nel] and BR1 derivatives [M][dim][NV]
    const double* d_vinv = nullptr;
    double *av_eps = nullptr, *av_grad = nullptr;
};

struct sisdc_ctx_s {
    sisdc_problem prob{};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;   // created when graphs are requested on the NULL stream
    std::vector<sisdc_level_s*> levels;
    // kernel timing (measurement hook): events around implicit-solve launches
    bool timing = false;
    int timing_level = -1;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_level;
    std::vector<int> ev_sweeps;
    size_t ev_used = 0;
    int* d_iters = nullptr;              // iterations of each timed launch
    size_t iters_cap = 0;
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    long long* d_stats = nullptr;
    double* d_part = nullptr;
    double* d_norms = nullptr;   // diagnostics scratch
    // solve log of one level (training data of the learned initial guess)
    int log_level = -1;
    double *log_r = nullptr, *log_dx = nullptr, *log_c = nullptr;
    int log_cap = 0;
    int* d_log_count = nullptr;
    int max_grid = 0;
    // Persson-Peraire artificial viscosity in f (sisdc_set_av)
    bool av_on = false;
    double av_kappa = 0.0, av_cs = 0.0;
    int av_comp = 0;
    // caller's allocator for the level work arrays (sisdc_set_allocator)
    sisdc_alloc_fn ualloc = nullptr;
    sisdc_release_fn urelease = nullptr;
    void* uuser = nullptr;
    std::string err;
    long long launches = 0;
    long long sweeps[8] = {0};
    // captured step
    cudaGraphExec_t gexec = nullptr;
    double* g_u = nullptr;
    double g_dt = 0.0;
    int g_ncycles = -1, g_start = -1, g_post = -1;
    long long g_launches = 0, g_sweeps[8] = {0};   // per replay of the captured step
};

namespace {

struct Fail {
    sisdc_status st;
};

void check(sisdc_ctx_s* c, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{SISDC_E_CUDA};
    }
}

sisdc_status fail(sisdc_ctx_s* c, sisdc_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

// nu_d of nu_tilde = nu_d + dt_m/2 lam_max^2: the physical diffusivity for
// convection-diffusion and Burgers, none for Euler, and for Navier-Stokes the
// largest of the momentum and heat diffusivities 4/3 mu / rho and
// gamma mu / (Pr rho) at the reference density
double nu_d(const sisdc_problem& p) {
    if (p.pde == SISDC_PDE_EULER) return 0.0;
    if (p.pde == SISDC_PDE_NS) return std::max(4.0 / 3.0, p.gamma / p.Pr) * p.mu / p.rho_ref;
    return p.nu;
}
// diffusivity of the nu L u term of f (the Navier-Stokes viscous term is separate)
double nu_phys(const sisdc_problem& p) { return p.pde == SISDC_PDE_EULER || p.pde == SISDC_PDE_NS ? 0.0 : p.nu; }
double kappa_ns(const sisdc_problem& p) {
    return p.pde == SISDC_PDE_NS ? p.mu * p.gamma / ((p.gamma - 1.0) * p.Pr) : 0.0;
}

double* Um(sisdc_level_s* lv, double* U, int m) { return U + (long long)m * lv->NV; }

// ---- kernel wrappers ---------------------------------------------------------
void k_conv(sisdc_level_s* lv, const double* u, double* out, double* lam, int mode = CONV_OUT,
            double* cache = nullptr, double* delta = nullptr) {
    sisdc_ctx_s* c = lv->ctx;
    ConvArgs a{};
    a.g = lv->geo;
    a.pde = c->prob.pde == SISDC_PDE_NS ? SISDC_PDE_EULER : c->prob.pde;   // the NS convective flux is Euler's
    a.gamma = c->prob.gamma;
    a.ax = c->prob.adv[0];
    a.ay = c->prob.adv[1];
    a.u = u;
    a.out = out;
    a.cache = cache;
    a.delta = delta;
    a.lam = lam;
    a.mode = mode;
    check(c, launch_conv(a, c->stream), "conv kernel");
    c->launches++;
}

void k_lap(sisdc_level_s* lv, const double* u, double* out, int mode, double* out2 = nullptr,
           const double* cc = nullptr, Coef cf = Coef{0.0, 0.0, nullptr}) {
    sisdc_ctx_s* c = lv->ctx;
    check(c, launch_traces(lv->geo, u, lv->trx, c->stream), "trace kernel");
    ApplyArgs a{};
    a.g = lv->geo;
    a.u = u;
    a.tr = lv->trx;
    a.out = out;
    a.out2 = out2;
    a.cc = cc;
    a.nu = nu_phys(c->prob);
    a.c = cf;
    a.mode = mode;
    check(c, launch_apply(a, c->stream), "SIPG apply kernel");
    c->launches += 2;
}

struct Terms {
    int n = 0;
    const double* in[MAXTERMS];
    Coef cf[MAXTERMS];
    void add(const double* p, double a0, double a2 = 0.0, const double* lam = nullptr) {
        in[n] = p;
        cf[n] = Coef{a0, a2, lam};
        ++n;
    }
};

void k_pcg(sisdc_level_s* lv, double* x, const Terms& t, Coef cimp, int prec = PCG_JACOBI) {
    sisdc_ctx_s* c = lv->ctx;
    PCGArgs a{};
    a.prec = prec;
    a.z = lv->cg_rf;
    a.g = lv->geo;
    a.x = x;
    a.r = lv->cg_r;
    a.p = lv->cg_p;
    a.Ap = lv->cg_Ap;
    a.trx = lv->trx;
    a.trp = lv->trp;
    a.nterms = t.n;
    for (int q = 0; q < t.n; ++q) {
        a.in[q] = t.in[q];
        a.coef[q] = t.cf[q];
    }
    a.cimp = cimp;
    a.part = c->d_part;
    a.bar_count = c->d_bar;
    a.bar_exit = c->d_bar + 1;
    a.err = c->d_err;
    a.stats = c->d_stats;
    a.rtol = c->prob.cg_rtol;
    a.maxit = c->prob.cg_maxit;
    a.iters_out = nullptr;
    check(c, launch_pcg(a, lv->pcg_grid, lv->pcg_block, c->stream), "PCG kernel");
    c->launches++;
}

void k_lin(sisdc_level_s* lv, double* out, const Terms& t, long long n = -1) {
    LinArgs a{};
    a.n = n < 0 ? lv->NV : n;
    a.nterms = t.n;
    for (int q = 0; q < t.n; ++q) {
        a.in[q] = t.in[q];
        a.coef[q] = t.cf[q];
    }
    a.out = out;
    check(lv->ctx, launch_lincomb(a, lv->ctx->stream), "lincomb kernel");
    lv->ctx->launches++;
}

void copy_d2d(sisdc_level_s* lv, double* dst, const double* src, long long n) {
    if (dst == src) return;
    check(lv->ctx, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, lv->ctx->stream),
          "device copy");
}

// transfer between lv (fine) and its coarser level
enum { T_INTERP = 0, T_PROJECT = 1, T_RESTRICT = 2, T_PROJECT_SPACE = 3 };
void k_transfer(sisdc_level_s* fine, int op, const double* in, double* out, int add) {
    sisdc_level_s* coarse = fine->ctx->levels[fine->index - 1];
    TransferArgs a{};
    a.dim = fine->desc.dim;
    a.ncomp = fine->ctx->prob.ncomp;
    a.nel = fine->nel;
    a.in = in;
    a.out = out;
    a.add = add;
    switch (op) {
        case T_INTERP:
            a.nqi = coarse->nq; a.nqo = fine->nq; a.Mi = coarse->M; a.Mo = fine->M;
            a.S = fine->d_Ix; a.Tt = fine->d_It;
            break;
        case T_PROJECT:
            a.nqi = fine->nq; a.nqo = coarse->nq; a.Mi = fine->M; a.Mo = coarse->M;
            a.S = fine->d_Px; a.Tt = fine->d_Pt;
            break;
        case T_RESTRICT:
            a.nqi = fine->nq; a.nqo = coarse->nq; a.Mi = fine->M; a.Mo = coarse->M;
            a.S = fine->d_Rx; a.Tt = fine->d_Rt;
            break;
        default:
            a.nqi = fine->nq; a.nqo = coarse->nq; a.Mi = 1; a.Mo = 1;
            a.S = fine->d_Px; a.Tt = fine->d_one;
            break;
    }
    if (fine->rx > 1 || fine->ry > 1) {
        a.rx = fine->rx;
        a.ry = fine->ry;
        a.c2f = op == T_INTERP;
        a.Sy = op == T_INTERP ? fine->d_Iy : op == T_RESTRICT ? fine->d_Ry : fine->d_Py;
        const sisdc_level_s* li = op == T_INTERP ? coarse : fine;
        const sisdc_level_s* lo = op == T_INTERP ? fine : coarse;
        a.nexi = li->desc.nel[0];
        a.neyi = li->desc.dim == 2 ? li->desc.nel[1] : 1;
        a.nexo = lo->desc.nel[0];
        a.neyo = lo->desc.dim == 2 ? lo->desc.nel[1] : 1;
    }
    check(fine->ctx, launch_transfer(a, fine->ctx->stream), "transfer kernel");
    fine->ctx->launches++;
}


// ---- method building blocks ----------------------------------------------------
// the artificial viscosity's share of nu_tilde per unit of lam_max: c_s h / P,
// h the smaller element side (0 without artificial viscosity)
double av_nu_lam(const sisdc_level_s* lv) {
    const sisdc_ctx_s* c = lv->ctx;
    if (!c->av_on) return 0.0;
    const double h = lv->desc.dim == 2 ? std::min(lv->geo.hx, lv->geo.hy) : lv->geo.hx;
    return c->av_cs * h / lv->desc.P;
}

// F_s += div(eps grad U_s) for the n states U_s, F_s (artificial viscosity of
// f, evaluated at the same states as the rest of f)
void av_add(sisdc_level_s* lv, const double* U, double* F, int n) {
    sisdc_ctx_s* c = lv->ctx;
    AvArgs a{};
    a.g = lv->geo;
    a.pde = c->prob.pde == SISDC_PDE_NS ? SISDC_PDE_EULER : c->prob.pde;
    a.gamma = c->prob.gamma;
    a.ax = c->prob.adv[0];
    a.ay = c->prob.adv[1];
    a.comp = c->av_comp;
    a.s0 = std::log10(1.0 / std::pow((double)lv->desc.P, 4));
    a.kappa = c->av_kappa;
    a.eps_scale = av_nu_lam(lv);
    a.vinv = lv->d_vinv;
    a.U = U;
    a.F = F;
    a.eps = lv->av_eps;
    a.grad = lv->av_grad;
    a.n = n;
    check(c, launch_av(a, c->stream), "artificial viscosity kernels");
    c->launches += 3;
}

// One cooperative launch of the persistent sweep kernel (sweep.cuh).
void run_sweep_kernel(sisdc_level_s* lv, int mode, const double* u0, double* U, const double* G, double dt,
                      int nsweeps, double* fout = nullptr) {
    sisdc_ctx_s* c = lv->ctx;
    SweepArgs a{};
    a.g = lv->geo;
    a.pde = c->prob.pde;
    a.gamma = c->prob.gamma;
    a.ax = c->prob.adv[0];
    a.ay = c->prob.adv[1];
    a.nu = nu_phys(c->prob);
    a.nu_d = nu_d(c->prob);
    a.nu_tilde_fix = c->prob.nu_tilde;
    a.nu_lam = av_nu_lam(lv);
    a.mu = c->prob.pde == SISDC_PDE_NS ? c->prob.mu : 0.0;
    a.kappa = kappa_ns(c->prob);
    a.FV = lv->FV;
    a.fout = fout;
    a.mode = mode;
    a.nsweeps = nsweeps;
    a.stages = c->prob.si_stages;
    a.M = lv->M;
    a.dt = dt;
    for (int m = 0; m < lv->M; ++m) a.dtau[m] = lv->tab.dtau[m];
    for (int k = 0; k < lv->M * lv->M; ++k) a.W[k] = lv->tab.wnn[k];
    a.u0 = u0;
    a.U = U;
    a.G = G;
    a.mix = lv->mix ? 1 : 0;
    a.F = lv->F; a.CC = lv->CC; a.LU = lv->LU; a.Qb = lv->Qb;
    a.c0 = lv->c0; a.dC = lv->dC; a.tmpc = lv->tmpc;
    a.r = lv->cg_r; a.p = lv->cg_p; a.p2 = lv->cg_p2; a.Ap = lv->cg_Ap; a.rf = lv->cg_rf;
    a.lam = lv->lam;
    a.part = c->d_part;
    a.partmax = c->d_part + 8 * (size_t)c->max_grid;
    a.bar_count = c->d_bar;
    a.bar_exit = c->d_bar + 1;
    a.err = c->d_err;
    a.stats = c->d_stats;
    a.rtol = c->prob.cg_rtol;
    a.maxit = c->prob.cg_maxit;
    a.epb = lv->sw_epb;
    a.stream = c->stream;
    a.iters_out = nullptr;
    if (c->log_r && lv->index == c->log_level && !lv->mix) {
        a.log_r = c->log_r;
        a.log_dx = c->log_dx;
        a.log_c = c->log_c;
        a.log_count = c->d_log_count;
        a.log_cap = c->log_cap;
    }
    const bool timed = c->timing && mode == SW_CORRECT && (c->timing_level < 0 || c->timing_level == lv->index);
    if (timed) {
        const size_t k = c->ev_used / 2;
        if (c->ev_used + 2 > c->ev.size()) {
            for (int q = 0; q < 2; ++q) {
                cudaEvent_t e;
                check(c, cudaEventCreate(&e), "event create");
                c->ev.push_back(e);
            }
        }
        if (k >= c->iters_cap) {
            const size_t cap = c->iters_cap ? 2 * c->iters_cap : 1024;
            int* p = nullptr;
            check(c, cudaStreamSynchronize(c->stream), "sync");
            check(c, cudaMalloc(&p, cap * sizeof(int)), "timing buffer");
            check(c, cudaMemset(p, 0, cap * sizeof(int)), "timing buffer");
            if (c->d_iters) {
                check(c, cudaMemcpy(p, c->d_iters, c->iters_cap * sizeof(int), cudaMemcpyDeviceToDevice), "copy");
                cudaFree(c->d_iters);
            }
            c->d_iters = p;
            c->iters_cap = cap;
        }
        a.iters_out = c->d_iters + k;
        check(c, cudaMemsetAsync(a.iters_out, 0, sizeof(int), c->stream), "memset");
        c->ev_level.push_back(lv->index);
        c->ev_sweeps.push_back(nsweeps);
        check(c, cudaEventRecord(c->ev[c->ev_used], c->stream), "event record");
    }
    check(c, launch_sweep(a, lv->sw_grid, lv->sw_block), "sweep kernel");
    if (timed) {
        check(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream), "event record");
        c->ev_used += 2;
    }
    c->launches++;
    // artificial viscosity: f at the states the kernel just evaluated f at
    // (every node, or the one state of SW_FEVAL); a correction launch runs
    // one sweep then (sweep())
    if (c->av_on) {
        if (mode == SW_FEVAL) av_add(lv, u0, fout, 1);
        else av_add(lv, U, lv->F, lv->M);
    }
}

// Caches f(U_m), c(U_m), L U_m, c(u0) and the spectral-radius slots of (u0, U).
void refresh(sisdc_level_s* lv, const double* u0, const double* U) {
    run_sweep_kernel(lv, SW_REFRESH, u0, const_cast<double*>(U), nullptr, 1.0, 0);
    lv->valid = true;
    lv->cache_u0 = u0;
    lv->cache_U = U;
}

void sweep_learned(sisdc_level_s* lv, const double* u0, double* U, const double* G, double dt, int nsweeps);

void sweep(sisdc_level_s* lv, const double* u0, double* U, const double* G, double dt, int nsweeps) {
    if (!lv->valid || lv->cache_u0 != u0 || lv->cache_U != U) refresh(lv, u0, U);
    if (nsweeps > 0) {
        if (lv->learned) sweep_learned(lv, u0, U, G, dt, nsweeps);
        else if (lv->ctx->av_on)            // f gains its viscosity term between sweeps
            for (int k = 0; k < nsweeps; ++k) run_sweep_kernel(lv, SW_CORRECT, u0, U, G, dt, 1);
        else run_sweep_kernel(lv, SW_CORRECT, u0, U, G, dt, nsweeps);
    }
    if (lv->index < 8) lv->ctx->sweeps[lv->index] += nsweeps;
    lv->valid = true;
    lv->cache_u0 = u0;
    lv->cache_U = U;
}

void predict(sisdc_level_s* lv, const double* u0, double* U, double dt) {
    run_sweep_kernel(lv, SW_PREDICT, u0, U, nullptr, dt, 0);
    if (lv->index < 8) lv->ctx->sweeps[lv->index]++;
    lv->valid = true;
    lv->cache_u0 = u0;
    lv->cache_U = U;
}

// The correction sweep of the persistent kernel (Algorithm 1 with the SI(1)
// / SI(2) right-hand sides, FP64) composed on the host from the
// single-operation kernels, with the learned initial guess before every
// implicit solve: x0 = u^{k-1}_m + z, z = MLP correction of the nodal
// residual of the warm start (sisdc_mlp_apply), then Jacobi-PCG from x0 to
// the same tolerance.  Spectral-radius slots and caches as in the kernel
// (old slots 0..M = lambda(u0), lambda(U_m) of the previous sweep; new
// slot m+1 = lambda(u^k_m)).  The network's scalar feature takes
// c = dt_m nu_tilde(lambda(u0)) (the solve itself uses its exact c).
void sweep_learned(sisdc_level_s* lv, const double* u0, double* U, const double* G, double dt, int nsweeps) {
    sisdc_ctx_s* c = lv->ctx;
    const sisdc_problem& pr = c->prob;
    const long long NV = lv->NV;
    const double nd = nu_d(pr), fix = pr.nu_tilde;
    double* lam_old = lv->lam;
    double* lam_new = lv->lam + MMAX + 1;
    auto coef_nut = [&](double dtm, double scale, const double* lam) {
        // scale * dt_m * nu_tilde(lam)
        if (fix > 0.0) return Coef{scale * dtm * fix, 0.0, nullptr};
        return Coef{scale * dtm * nd, scale * 0.5 * dtm * dtm, lam};
    };
    for (int k = 0; k < nsweeps; ++k) {
        double lam0 = 0.0;
        check(c, cudaMemcpyAsync(&lam0, lam_old, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "lambda read");
        check(c, cudaStreamSynchronize(c->stream), "sync");
        check(c, launch_quad(lv->F, 0, lv->Qb, lv->tab.wnn.data(), lv->M, dt, NV, c->stream), "quad kernel");
        c->launches++;
        for (int m = 0; m < lv->M; ++m) {
            const double dtm = dt * lv->tab.dtau[m];
            const double* up = m ? Um(lv, U, m - 1) : u0;
            double* um = Um(lv, U, m);
            const double* Qm = lv->Qb + (long long)m * NV;
            const double* Gm = G ? G + (long long)m * NV : nullptr;
            double* LUm = lv->LU + (long long)m * NV;
            double* CCm = lv->CC + (long long)m * NV;
            if (dtm == 0.0) {                                    // Lobatto t_1 = t_0
                Terms t;
                t.add(up, 1.0);
                t.add(Qm, 1.0);
                if (Gm) t.add(Gm, 1.0);
                k_lin(lv, um, t);
            } else {
                const double* lcur = m == 0 ? lam_old : lam_new + m;   // lambda(u^k_{m-1})
                const Coef cnew = coef_nut(dtm, 1.0, lcur);
                const double cfeat = dtm * (fix > 0.0 ? fix : nd + 0.5 * dtm * lam0 * lam0);
                Terms t1;
                t1.add(up, 1.0);
                t1.add(Qm, 1.0);
                if (Gm) t1.add(Gm, 1.0);
                const Coef cold = coef_nut(dtm, -1.0, lam_old + m);
                t1.add(LUm, cold.a0, cold.a2, cold.lam);
                Terms t2 = t1;
                if (m > 0) t1.add(lv->dC, dtm);
                // stage 1: r0 = b - (x0 - c L x0) with the cached L x0, guess, solve
                {
                    Terms tr = t1;
                    tr.add(um, -1.0);
                    tr.add(LUm, cnew.a0, cnew.a2, cnew.lam);
                    k_lin(lv, lv->cg_r, tr);
                    const sisdc_status st = sisdc_mlp_apply(lv->learned, lv->cg_r, cfeat, um, 1);
                    if (st != SISDC_OK) throw Fail{st};
                    k_pcg(lv, um, t1, cnew);
                }
                if (pr.si_stages == 2) {
                    k_conv(lv, um, lv->tmpc, nullptr);           // c(u^(1))
                    t2.add(lv->tmpc, dtm);
                    t2.add(CCm, -dtm);                            // c(u^{k-1}_m)
                    k_lap(lv, um, lv->cg_p, APPLY_LAP);           // L x0 (x0 = u^(1))
                    Terms tr = t2;
                    tr.add(um, -1.0);
                    tr.add(lv->cg_p, cnew.a0, cnew.a2, cnew.lam);
                    k_lin(lv, lv->cg_r, tr);
                    const sisdc_status st = sisdc_mlp_apply(lv->learned, lv->cg_r, cfeat, um, 1);
                    if (st != SISDC_OK) throw Fail{st};
                    k_pcg(lv, um, t2, cnew);
                }
            }
            // node end: f(u^k_m), c(u^k_m) with its change, L u^k_m, lambda(u^k_m)
            run_sweep_kernel(lv, SW_FEVAL, um, lv->U, nullptr, 1.0, 0, lv->F + (long long)m * NV);
            check(c, cudaMemsetAsync(lam_new + m + 1, 0, sizeof(double), c->stream), "memset");
            k_conv(lv, um, nullptr, lam_new + m + 1, CONV_DELTA, CCm, lv->dC);
            k_lap(lv, um, LUm, APPLY_LAP);
        }
        check(c, cudaMemcpyAsync(lam_old + 1, lam_new + 1, lv->M * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream), "lambda slots");
    }
}

// r = G - F^nn(U) (G may be null); needs valid caches
void residual(sisdc_level_s* lv, const double* u0, const double* U, const double* G, double dt, double* r) {
    sisdc_ctx_s* c = lv->ctx;
    if (!lv->valid || lv->cache_u0 != u0 || lv->cache_U != U) refresh(lv, u0, U);
    check(c, launch_quad(lv->F, 0, lv->Qb, lv->tab.wnn.data(), lv->M, dt, lv->NV, c->stream), "quad kernel");
    check(c, launch_fnn(u0, U, lv->Qb, G, r, lv->M, lv->NV, 1, c->stream), "fnn kernel");
    c->launches += 2;
}

struct LevelPtrs {
    std::vector<const double*> u0;
    std::vector<double*> U;
};

// Algorithm 2 on levels 0..top-1 (top-1 acts as the finest level, g = 0).
void vcycle(sisdc_ctx_s* c, LevelPtrs& P, int top, double dt, int Nc) {
    std::vector<sisdc_level_s*>& L = c->levels;
    for (int l = top - 1; l >= 1; --l) {
        sisdc_level_s* f = L[l];
        sisdc_level_s* cl = L[l - 1];
        const double* Gf = (l == top - 1) ? nullptr : f->G;
        sweep(f, P.u0[l], P.U[l], Gf, dt, 1);                                  // pre-sweep
        residual(f, P.u0[l], P.U[l], Gf, dt, f->R);                            // r_l = g_l - F_l(u_l)
        k_transfer(f, T_PROJECT, P.U[l], P.U[l - 1], 0);                        // v_{l-1} = P u_l
        copy_d2d(cl, cl->V, P.U[l - 1], (long long)cl->M * cl->NV);
        refresh(cl, P.u0[l - 1], P.U[l - 1]);
        check(c, launch_quad(cl->F, 0, cl->Qb, cl->tab.wnn.data(), cl->M, dt, cl->NV, c->stream), "quad kernel");
        check(c, launch_fnn(P.u0[l - 1], P.U[l - 1], cl->Qb, nullptr, cl->G, cl->M, cl->NV, 0, c->stream),
              "fnn kernel");
        c->launches += 2;
        k_transfer(f, T_RESTRICT, f->R, cl->G, 1);                             // g_{l-1} += R r_l
    }
    sweep(L[0], P.u0[0], P.U[0], top > 1 ? L[0]->G : nullptr, dt, Nc);        // coarse solve
    for (int l = 1; l < top; ++l) {
        sisdc_level_s* f = L[l];
        sisdc_level_s* cl = L[l - 1];
        Terms d;
        d.add(P.U[l - 1], 1.0);
        d.add(cl->V, -1.0);
        k_lin(cl, cl->R, d, (long long)cl->M * cl->NV);                         // u_{l-1} - v_{l-1}
        k_transfer(f, T_INTERP, cl->R, P.U[l], 1);                              // u_l += I(...)
        f->valid = false;
        if (l < top - 1) sweep(f, P.u0[l], P.U[l], f->G, dt, 1);              // post-sweep
    }
}

void start_strategy(sisdc_ctx_s* c, LevelPtrs& P, double dt, int start) {
    std::vector<sisdc_level_s*>& L = c->levels;
    const int nl = (int)L.size();
    if (start == SISDC_START_CASCADE || start == SISDC_START_FMG1) {
        predict(L[0], P.u0[0], P.U[0], dt);
        sweep(L[0], P.u0[0], P.U[0], nullptr, dt, 1);
        if (nl > 1) {
            k_transfer(L[1], T_INTERP, P.U[0], P.U[1], 0);
            L[1]->valid = false;
        }
        for (int l = 1; l < nl - 1; ++l) {
            if (start == SISDC_START_FMG1)                 // C_fmg V-cycles per added level
                for (int k = 0; k < std::max(1, c->prob.fmg_cycles); ++k) vcycle(c, P, l + 1, dt, c->prob.Nc);
            else sweep(L[l], P.u0[l], P.U[l], nullptr, dt, 1);
            k_transfer(L[l + 1], T_INTERP, P.U[l], P.U[l + 1], 0);
            L[l + 1]->valid = false;
        }
    } else if (start == SISDC_START_PREDICTOR) {
        for (int l = 0; l < nl; ++l) predict(L[l], P.u0[l], P.U[l], dt);
    } else {
        for (int l = 0; l < nl; ++l) {
            for (int m = 0; m < L[l]->M; ++m) copy_d2d(L[l], Um(L[l], P.U[l], m), P.u0[l], L[l]->NV);
            L[l]->valid = false;
        }
    }
}

void enqueue_step(sisdc_ctx_s* c, double* d_u, double dt, int ncycles, int start, int post) {
    std::vector<sisdc_level_s*>& L = c->levels;
    const int nl = (int)L.size();
    sisdc_level_s* fine = L[nl - 1];
    LevelPtrs P;
    P.u0.resize(nl);
    P.U.resize(nl);
    copy_d2d(fine, fine->u0, d_u, fine->NV);
    for (int l = 0; l < nl; ++l) {
        P.u0[l] = L[l]->u0;
        P.U[l] = L[l]->U;
        L[l]->valid = false;
    }
    for (int l = nl - 1; l >= 1; --l) k_transfer(L[l], T_PROJECT_SPACE, L[l]->u0, L[l - 1]->u0, 0);
    if (nl == 1) {
        predict(fine, fine->u0, fine->U, dt);
        sweep(fine, fine->u0, fine->U, nullptr, dt, ncycles);
    } else {
        start_strategy(c, P, dt, start);
        for (int k = 0; k < ncycles; ++k) vcycle(c, P, nl, dt, c->prob.Nc);
        if (post) sweep(fine, fine->u0, fine->U, nullptr, dt, 1);
    }
    copy_d2d(fine, d_u, Um(fine, fine->U, fine->M - 1), fine->NV);
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
// Level work memory: the caller's allocator when one is set, else cudaMalloc.
static cudaError_t level_alloc(sisdc_ctx_s* c, double** p, size_t bytes) {
    *p = nullptr;
    if (!c->ualloc) return cudaMalloc(reinterpret_cast<void**>(p), bytes);
    void* q = c->ualloc(bytes, c->stream, c->uuser);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<unsigned long long>(q) % 256 != 0) {
        c->urelease(q, bytes, c->stream, c->uuser);
        return cudaErrorMisalignedAddress;
    }
    *p = static_cast<double*>(q);
    return cudaSuccess;
}

static void level_free(sisdc_ctx_s* c, double* p, size_t bytes) {
    if (!p) return;
    if (c->urelease) c->urelease(p, bytes, c->stream, c->uuser);
    else cudaFree(p);
}

static void level_free_all(sisdc_ctx_s* c, sisdc_level_s* lv) {
    level_free(c, lv->d_tab, lv->tab_bytes);
    level_free(c, lv->d_mem, lv->mem_bytes);
    lv->d_tab = lv->d_mem = nullptr;
}

extern "C" {

sisdc_status sisdc_create(const sisdc_problem* prob, void* cuda_stream, sisdc_ctx* out) {
    if (!prob || !out) return SISDC_E_ARG;
    *out = nullptr;
    const int nc_expect = prob->pde == SISDC_PDE_CONVDIFF ? 1 : prob->pde == SISDC_PDE_BURGERS ? 2
                          : (prob->pde == SISDC_PDE_EULER || prob->pde == SISDC_PDE_NS) ? 4 : -1;
    if (nc_expect < 0 || prob->ncomp != nc_expect) return SISDC_E_ARG;
    if (prob->si_stages != 1 && prob->si_stages != 2) return SISDC_E_ARG;
    if (prob->precision != SISDC_FP64 && prob->precision != SISDC_MIXED) return SISDC_E_ARG;
    if (prob->mixed_levels < 0) return SISDC_E_ARG;
    if (!(prob->cg_rtol > 0.0) || prob->cg_maxit < 1 || prob->Nc < 0) return SISDC_E_ARG;
    if ((prob->pde == SISDC_PDE_EULER || prob->pde == SISDC_PDE_NS) && !(prob->gamma > 1.0)) return SISDC_E_ARG;
    if (prob->pde == SISDC_PDE_NS && !(prob->mu > 0.0 && prob->Pr > 0.0 && prob->rho_ref > 0.0)) return SISDC_E_ARG;
    if (prob->projection != 0 && prob->projection != 1) return SISDC_E_ARG;
    if (prob->fmg_cycles < 0) return SISDC_E_ARG;
    if (prob->form != 0 && prob->form != 1) return SISDC_E_ARG;
    if (prob->nu < 0.0) return SISDC_E_ARG;
    if (!(prob->nu_tilde >= 0.0) || !std::isfinite(prob->nu_tilde)) return SISDC_E_ARG;
    sisdc_ctx_s* c = new sisdc_ctx_s();
    c->prob = *prob;
    c->stream = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && prob->use_graph && cuda_stream == nullptr) {
        // the legacy stream cannot be captured; a blocking stream keeps the
        // legacy stream's ordering with respect to other work
        e = cudaStreamCreate(&c->own_stream);
        c->stream = c->own_stream;
    }
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    c->max_grid = 32 * (nsm > 0 ? nsm : 160);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, ST_N * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_part, (8 + MMAX + 1) * (size_t)c->max_grid * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_norms, norms_scratch_doubles(prob->ncomp) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_log_count, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_log_count, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, ST_N * sizeof(long long));
    if (e != cudaSuccess) {
        sisdc_destroy(c);
        return e == cudaErrorMemoryAllocation ? SISDC_E_OOM : SISDC_E_CUDA;
    }
    *out = c;
    return SISDC_OK;
}

void sisdc_destroy(sisdc_ctx c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    cudaFree(c->d_iters);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (sisdc_level_s* lv : c->levels) {
        level_free_all(c, lv);
        delete lv;
    }
    cudaFree(c->d_bar);
    cudaFree(c->d_err);
    cudaFree(c->d_stats);
    cudaFree(c->d_part);
    cudaFree(c->d_norms);
    cudaFree(c->d_log_count);
    delete c;
}

sisdc_status sisdc_set_allocator(sisdc_ctx c, sisdc_alloc_fn alloc, sisdc_release_fn release, void* user) {
    if (!c) return SISDC_E_ARG;
    if ((alloc == nullptr) != (release == nullptr)) return fail(c, SISDC_E_ARG, "allocator: alloc and release go together");
    if (!c->levels.empty()) return fail(c, SISDC_E_STATE, "allocator must be set before the first level");
    c->ualloc = alloc;
    c->urelease = release;
    c->uuser = alloc ? user : nullptr;
    return SISDC_OK;
}

sisdc_status sisdc_set_av(sisdc_ctx c, double d_s, double c_s, int comp) {
    if (!c) return SISDC_E_ARG;
    if (!c->levels.empty()) return fail(c, SISDC_E_STATE, "artificial viscosity must be set before the first level");
    if (c_s == 0.0) {
        c->av_on = false;
        return SISDC_OK;
    }
    if (!(d_s > 0.0) || !(c_s > 0.0) || !std::isfinite(d_s) || !std::isfinite(c_s))
        return fail(c, SISDC_E_ARG, "artificial viscosity: d_s and c_s must be positive and finite");
    if (comp < 0 || comp >= c->prob.ncomp) return fail(c, SISDC_E_ARG, "artificial viscosity: bad sensor component");
    c->av_on = true;
    c->av_kappa = d_s;
    c->av_cs = c_s;
    c->av_comp = comp;
    return SISDC_OK;
}

sisdc_status sisdc_create_level(sisdc_ctx c, const sisdc_level_desc* d, sisdc_level* out) {
    if (!c || !d || !out) return SISDC_E_ARG;
    *out = nullptr;
    if (d->dim != 1 && d->dim != 2) return fail(c, SISDC_E_ARG, "dim must be 1 or 2");
    if (d->dim == 1 && c->prob.pde != SISDC_PDE_CONVDIFF) return fail(c, SISDC_E_ARG, "1D supports convection-diffusion only");
    if ((long long)d->nel[0] * (d->dim == 2 ? d->nel[1] : 1) > (1LL << 30)) return fail(c, SISDC_E_ARG, "too many elements");
    const int lidx = (int)c->levels.size();
    const bool lmix = c->prob.precision == SISDC_MIXED &&
                      (c->prob.mixed_levels == 0 || (lidx < 31 && ((c->prob.mixed_levels >> lidx) & 1)));
    // degrees up to 15 for 1D convection-diffusion in FP64, up to 8 otherwise
    const int pmax = (d->dim == 1 && c->prob.pde == SISDC_PDE_CONVDIFF && !lmix) ? 15 : 8;
    if (d->P < 1 || d->P > pmax) return fail(c, SISDC_E_ARG, "P must be in 1..8 (1..15 for 1D convection-diffusion in FP64)");
    if (d->M < 1 || d->M > MMAX) return fail(c, SISDC_E_ARG, "M must be in 1..8");
    if (d->nodes != SISDC_RADAU_RIGHT && d->nodes != SISDC_LOBATTO) return fail(c, SISDC_E_ARG, "bad node kind");
    if (d->nodes == SISDC_LOBATTO && d->M < 2) return fail(c, SISDC_E_ARG, "Lobatto needs M >= 2");
    const int ney = d->dim == 2 ? d->nel[1] : 1;
    if (d->nel[0] < 1 || ney < 1) return fail(c, SISDC_E_ARG, "nel must be >= 1");
    if (!(d->hi[0] > d->lo[0]) || (d->dim == 2 && !(d->hi[1] > d->lo[1]))) return fail(c, SISDC_E_ARG, "empty box");
    if ((int)c->levels.size() >= 8) return fail(c, SISDC_E_ARG, "at most 8 levels");
    if (lmix && (d->dim != 2 || d->P < 3))
        return fail(c, SISDC_E_ARG, "mixed precision supports 2D levels with P >= 3");
    if (!c->levels.empty()) {
        const sisdc_level_desc& p = c->levels.back()->desc;
        const bool gx = d->nel[0] == p.nel[0] || d->nel[0] == 2 * p.nel[0];
        const bool gy = d->dim == 1 || d->nel[1] == p.nel[1] || d->nel[1] == 2 * p.nel[1];
        if (p.dim != d->dim || !gx || !gy || p.nodes != d->nodes || p.lo[0] != d->lo[0] || p.hi[0] != d->hi[0] ||
            (d->dim == 2 && (p.lo[1] != d->lo[1] || p.hi[1] != d->hi[1])))
            return fail(c, SISDC_E_ARG,
                        "levels must share dim, box and node kind; element grids equal or 2:1 per direction");
        if (p.P > d->P || p.M > d->M) return fail(c, SISDC_E_ARG, "levels must be added coarse to fine");
    }
    sisdc_level_s* lv = new sisdc_level_s();
    lv->ctx = c;
    lv->index = lidx;
    lv->mix = lmix;
    lv->desc = *d;
    if (d->dim == 1) { lv->desc.nel[1] = 1; lv->desc.lo[1] = 0.0; lv->desc.hi[1] = 1.0; }
    if (!build_level_tables(d->P, d->M, d->nodes == SISDC_LOBATTO, &lv->tab)) {
        delete lv;
        return fail(c, SISDC_E_ARG, "table construction failed");
    }
    lv->nq = d->P + 1;
    lv->nqy = d->dim == 2 ? lv->nq : 1;
    lv->Q = lv->nq * lv->nqy;
    lv->M = d->M;
    lv->nel = d->nel[0] * ney;
    lv->N = (long long)lv->nel * lv->Q;
    lv->NV = lv->N * c->prob.ncomp;
    const double hx = (d->hi[0] - d->lo[0]) / d->nel[0];
    const double hy = d->dim == 2 ? (d->hi[1] - d->lo[1]) / ney : 1.0;
    const int nq = lv->nq;
    const double taux = 2.0 * nq * nq / hx, tauy = 2.0 * nq * nq / hy;
    std::vector<double> htab(2 * nq * nq + 3 * nq);
    for (int k = 0; k < nq * nq; ++k) { htab[k] = lv->tab.D[k]; htab[nq * nq + k] = lv->tab.K[k]; }
    for (int i = 0; i < nq; ++i) {
        htab[2 * nq * nq + i] = lv->tab.w[i];
        double dx = (2.0 / hx) * lv->tab.Kdiag[i], dy = (2.0 / hy) * lv->tab.Kdiag[i];
        if (i == nq - 1) { dx += -2.0 * lv->tab.DPP / hx + taux; dy += -2.0 * lv->tab.DPP / hy + tauy; }
        if (i == 0) { dx += 2.0 * lv->tab.D00 / hx + taux; dy += 2.0 * lv->tab.D00 / hy + tauy; }
        htab[2 * nq * nq + nq + i] = dx;
        htab[2 * nq * nq + 2 * nq + i] = dy;
    }
    // element-wise fast-diagonalisation tables (x, then y): S_x, lam_x, S_y, lam_y
    const size_t off_fds = htab.size();
    htab.resize(off_fds + 2 * (nq * nq + nq));
    if (!fds_tables(d->P, hx, htab.data() + off_fds, htab.data() + off_fds + nq * nq) ||
        !fds_tables(d->P, hy, htab.data() + off_fds + nq * nq + nq, htab.data() + off_fds + 2 * nq * nq + nq)) {
        delete lv;
        return fail(c, SISDC_E_ARG, "table construction failed");
    }
    // nodal-to-modal matrix of the artificial-viscosity sensor
    const size_t off_vinv = htab.size();
    if (c->av_on) {
        htab.resize(off_vinv + nq * nq);
        if (!modal_matrix(d->P, htab.data() + off_vinv)) {
            delete lv;
            return fail(c, SISDC_E_ARG, "table construction failed");
        }
    }
    // transfers to the coarser level
    std::vector<double> ttab;
    size_t off_Ix = 0, off_Px = 0, off_Rx = 0, off_It = 0, off_Pt = 0, off_Rt = 0, off_one = 0;
    size_t off_Iy = 0, off_Py = 0, off_Ry = 0;
    if (lv->index > 0) {
        sisdc_level_s* cl = c->levels.back();
        const std::vector<double>& xf = lv->tab.gll;
        const std::vector<double>& xc = cl->tab.gll;
        std::vector<double> Ix = lagrange_matrix(xc, xf);   // (nqf x nqc)
        // solution projection (nqc x nqf): embedded interpolation, or the L2 projection
        std::vector<double> Px = c->prob.projection == 1 ? l2_projection_matrix(d->P, cl->desc.P)
                                                         : lagrange_matrix(xf, xc);
        std::vector<double> Rx(cl->nq * nq);
        for (int a = 0; a < cl->nq; ++a)
            for (int b = 0; b < nq; ++b) Rx[a * nq + b] = Ix[b * cl->nq + a] * lv->tab.w[b] / cl->tab.w[a];
        std::vector<double> It = lagrange_matrix(cl->tab.tau, lv->tab.tau);   // (Mf x Mc)
        std::vector<double> Pt = lagrange_matrix(lv->tab.tau, cl->tab.tau);   // (Mc x Mf)
        std::vector<double> Rt(cl->M * lv->M);
        for (int a = 0; a < cl->M; ++a)
            for (int b = 0; b < lv->M; ++b) Rt[a * lv->M + b] = It[b * cl->M + a];
        if (c->prob.form == 1) {
            // zero-to-node form (Sec. 4.5): the levels solve F^0n(u) = g^0n + C^0n dH with
            // F^0n = C^0n F^nn, i.e. the incremental equations with g^nn = (C^0n)^-1 g^0n;
            // the FAS restriction of the residual becomes (C_c^0n)^-1 R_t C_f^0n
            const int Mf = lv->M, Mc = cl->M;
            std::vector<double> RC(Mc * Mf);                    // R_t C_f: suffix sums over the fine index
            for (int a = 0; a < Mc; ++a) {
                double s = 0.0;
                for (int b = Mf - 1; b >= 0; --b) {
                    s += Rt[a * Mf + b];
                    RC[a * Mf + b] = s;
                }
            }
            for (int a = Mc - 1; a >= 0; --a)                   // (C_c)^-1: first differences over a
                for (int b = 0; b < Mf; ++b) Rt[a * Mf + b] = RC[a * Mf + b] - (a > 0 ? RC[(a - 1) * Mf + b] : 0.0);
        }
        auto push = [&](const std::vector<double>& v) { size_t o = ttab.size(); ttab.insert(ttab.end(), v.begin(), v.end()); return o; };
        lv->rx = d->nel[0] / cl->desc.nel[0];
        lv->ry = d->dim == 2 ? d->nel[1] / cl->desc.nel[1] : 1;
        if (lv->rx > 1 || lv->ry > 1) {
            // 2:1 h-coarsening in at least one direction: child matrices per direction
            std::vector<double> Ih, Ph, Rh;
            h_transfer_matrices(d->P, cl->desc.P, c->prob.projection == 1, &Ih, &Ph, &Rh);
            off_Ix = push(lv->rx > 1 ? Ih : Ix); off_Px = push(lv->rx > 1 ? Ph : Px); off_Rx = push(lv->rx > 1 ? Rh : Rx);
            off_Iy = push(lv->ry > 1 ? Ih : Ix); off_Py = push(lv->ry > 1 ? Ph : Px); off_Ry = push(lv->ry > 1 ? Rh : Rx);
        } else {
            off_Ix = push(Ix); off_Px = push(Px); off_Rx = push(Rx);
        }
        off_It = push(It); off_Pt = push(Pt); off_Rt = push(Rt);
        off_one = push(std::vector<double>{1.0});
    }
    const size_t ntab = htab.size() + ttab.size();
    lv->tab_bytes = ntab * sizeof(double);
    cudaError_t e = level_alloc(c, &lv->d_tab, lv->tab_bytes);
    // stream-ordered copies: memory of a caller's caching allocator may still
    // be in use by earlier work on the context stream
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lv->d_tab, htab.data(), htab.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !ttab.empty())
        e = cudaMemcpyAsync(lv->d_tab + htab.size(), ttab.data(), ttab.size() * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    // work arrays
    const long long NV = lv->NV, MV = (long long)lv->M * NV;
    const long long ntr = (long long)c->prob.ncomp * lv->nel * 2 * d->dim * 2 * nq;
    const long long nfv = c->prob.pde == SISDC_PDE_NS ? 6 * lv->N : 0;
    const long long nav = c->av_on ? (long long)lv->M * lv->nel + (long long)d->dim * MV : 0;
    const long long total = 8 * MV + 2 * NV + 3 * NV + 4 * NV + 2 * ntr + 2 * (MMAX + 1) + nfv + nav;
    lv->mem_bytes = total * sizeof(double);
    if (e == cudaSuccess) e = level_alloc(c, &lv->d_mem, lv->mem_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(lv->d_mem, 0, lv->mem_bytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        level_free_all(c, lv);
        delete lv;
        return fail(c, e == cudaErrorMemoryAllocation ? SISDC_E_OOM
                       : e == cudaErrorMisalignedAddress ? SISDC_E_ARG : SISDC_E_CUDA,
                    std::string("level allocation: ") +
                        (e == cudaErrorMisalignedAddress ? "allocator returned memory not 256-byte aligned"
                                                          : cudaGetErrorString(e)));
    }
    double* p = lv->d_mem;
    auto take = [&](long long n) { double* q = p; p += n; return q; };
    lv->U = take(MV); lv->F = take(MV); lv->CC = take(MV); lv->LU = take(MV);
    lv->Qb = take(MV); lv->G = take(MV); lv->V = take(MV); lv->R = take(MV);
    lv->u0 = take(NV); lv->c0 = take(NV);
    lv->dC = take(NV); lv->tmpc = take(NV); lv->cg_r = take(NV);
    lv->cg_p = take(NV); lv->cg_Ap = take(NV); lv->cg_p2 = take(NV); lv->cg_rf = take(NV);
    lv->trx = take(ntr); lv->trp = take(ntr);
    lv->lam = take(2 * (MMAX + 1));
    lv->FV = nfv ? take(nfv) : nullptr;
    if (c->av_on) {
        lv->av_eps = take((long long)lv->M * lv->nel);
        lv->av_grad = take((long long)d->dim * MV);
        lv->d_vinv = lv->d_tab + off_vinv;
    }
    if (lv->index > 0) {
        double* t = lv->d_tab + htab.size();
        lv->d_Ix = t + off_Ix; lv->d_Px = t + off_Px; lv->d_Rx = t + off_Rx;
        lv->d_It = t + off_It; lv->d_Pt = t + off_Pt; lv->d_Rt = t + off_Rt; lv->d_one = t + off_one;
        lv->d_Iy = t + off_Iy; lv->d_Py = t + off_Py; lv->d_Ry = t + off_Ry;
    }
    Geo& g = lv->geo;
    g.dim = d->dim; g.nq = nq; g.nqy = lv->nqy; g.q = lv->Q;
    g.nex = d->nel[0]; g.ney = ney; g.nel = lv->nel; g.ncomp = c->prob.ncomp;
    g.N = lv->N; g.hx = hx; g.hy = hy; g.taux = taux; g.tauy = tauy;
    g.D = lv->d_tab; g.K = lv->d_tab + nq * nq; g.w = lv->d_tab + 2 * nq * nq;
    g.dline_x = g.w + nq; g.dline_y = g.w + 2 * nq;
    g.fds = lv->d_tab + off_fds;
    g.sx = 2.0 / hx; g.sy = 2.0 / hy; g.ihx = 1.0 / hx; g.ihy = 1.0 / hy;
    g.liftLx = g.sx / lv->tab.w[0]; g.liftRx = g.sx / lv->tab.w[nq - 1];
    g.liftLy = g.sy / lv->tab.w[0]; g.liftRy = g.sy / lv->tab.w[nq - 1];
    lv->pcg_grid = pcg_grid(g, &lv->pcg_block);
    lv->sw_grid = sweep_config(g, c->prob.pde, lv->mix, &lv->sw_epb, &lv->sw_block);
    if (lv->pcg_grid < 1 || lv->pcg_grid > c->max_grid || lv->sw_grid < 1 || lv->sw_grid > c->max_grid) {
        level_free_all(c, lv);
        delete lv;
        return fail(c, SISDC_E_CUDA, "cooperative PCG launch configuration unavailable");
    }
    c->levels.push_back(lv);
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    *out = lv;
    return SISDC_OK;
}

sisdc_status sisdc_level_info(sisdc_level lv, int* ncomp, long long* nodes, int* M) {
    if (!lv) return SISDC_E_ARG;
    if (ncomp) *ncomp = lv->ctx->prob.ncomp;
    if (nodes) *nodes = lv->N;
    if (M) *M = lv->M;
    return SISDC_OK;
}

sisdc_status sisdc_level_coords(sisdc_level lv, double* hx_out, double* hy_out) {
    if (!lv || !hx_out) return SISDC_E_ARG;
    const sisdc_level_desc& d = lv->desc;
    const double hx = lv->geo.hx, hy = lv->geo.hy;
    for (int e = 0; e < lv->nel; ++e) {
        const int ex = e % d.nel[0], ey = e / d.nel[0];
        for (int j = 0; j < lv->nqy; ++j)
            for (int i = 0; i < lv->nq; ++i) {
                const long long k = (long long)e * lv->Q + j * lv->nq + i;
                hx_out[k] = d.lo[0] + (ex + (lv->tab.gll[i] + 1.0) / 2.0) * hx;
                if (hy_out) hy_out[k] = d.dim == 2 ? d.lo[1] + (ey + (lv->tab.gll[j] + 1.0) / 2.0) * hy : 0.0;
            }
    }
    return SISDC_OK;
}

sisdc_status sisdc_level_tables(sisdc_level lv, double* tau, double* wnn, double* gll, double* w, double* D) {
    if (!lv) return SISDC_E_ARG;
    if (tau) std::memcpy(tau, lv->tab.tau.data(), lv->M * sizeof(double));
    if (wnn) std::memcpy(wnn, lv->tab.wnn.data(), lv->M * lv->M * sizeof(double));
    if (gll) std::memcpy(gll, lv->tab.gll.data(), lv->nq * sizeof(double));
    if (w) std::memcpy(w, lv->tab.w.data(), lv->nq * sizeof(double));
    if (D) std::memcpy(D, lv->tab.D.data(), lv->nq * lv->nq * sizeof(double));
    return SISDC_OK;
}

#define SISDC_TRY(ctx, body)                                   \
    try {                                                      \
        body;                                                  \
    } catch (const Fail& f_) {                                 \
        return f_.st;                                          \
    } catch (...) {                                            \
        return fail(ctx, SISDC_E_CUDA, "unexpected host error"); \
    }                                                          \
    return SISDC_OK;

sisdc_status sisdc_apply_conv(sisdc_level lv, const double* u, double* out) {
    if (!lv || !u || !out) return SISDC_E_ARG;
    SISDC_TRY(lv->ctx, k_conv(lv, u, out, nullptr));
}

sisdc_status sisdc_apply_lap(sisdc_level lv, const double* u, double* out) {
    if (!lv || !u || !out) return SISDC_E_ARG;
    SISDC_TRY(lv->ctx, k_lap(lv, u, out, APPLY_LAP));
}

sisdc_status sisdc_apply_f(sisdc_level lv, const double* u, double* out) {
    if (!lv || !u || !out) return SISDC_E_ARG;
    sisdc_ctx_s* c = lv->ctx;
    try {
        run_sweep_kernel(lv, SW_FEVAL, u, lv->U, nullptr, 1.0, 0, out);
        lv->valid = false;
        check(c, cudaGetLastError(), "f evaluation");
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

static sisdc_status solve_prec(sisdc_level lv, double cval, const double* rhs, double* x, int* iters, int prec) {
    sisdc_ctx_s* c = lv->ctx;
    try {
        long long before = 0;
        if (iters) {
            check(c, cudaStreamSynchronize(c->stream), "sync");
            check(c, cudaMemcpy(&before, c->d_stats + ST_ITERS, sizeof(long long), cudaMemcpyDeviceToHost), "stats");
        }
        Terms t;
        t.add(rhs, 1.0);
        k_pcg(lv, x, t, Coef{cval, 0.0, nullptr}, prec);
        if (iters) {
            long long after = 0;
            check(c, cudaStreamSynchronize(c->stream), "sync");
            check(c, cudaMemcpy(&after, c->d_stats + ST_ITERS, sizeof(long long), cudaMemcpyDeviceToHost), "stats");
            *iters = (int)(after - before);
        }
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_solve(sisdc_level lv, double cval, const double* rhs, double* x, int* iters) {
    if (!lv || !rhs || !x || !(cval >= 0.0)) return SISDC_E_ARG;
    return solve_prec(lv, cval, rhs, x, iters, PCG_JACOBI);
}

sisdc_status sisdc_solve_fds(sisdc_level lv, double cval, const double* rhs, double* x, int* iters) {
    if (!lv || !rhs || !x || !(cval >= 0.0)) return SISDC_E_ARG;
    return solve_prec(lv, cval, rhs, x, iters, PCG_FDS);
}

sisdc_status sisdc_predict(sisdc_level lv, const double* u0, double* U, double dt) {
    if (!lv || !u0 || !U || !(dt > 0.0)) return SISDC_E_ARG;
    SISDC_TRY(lv->ctx, predict(lv, u0, U, dt));
}

sisdc_status sisdc_sweep(sisdc_level lv, const double* u0, double* U, const double* g, double dt, int nsweeps) {
    if (!lv || !u0 || !U || !(dt > 0.0) || nsweeps < 0) return SISDC_E_ARG;
    lv->valid = false;   // the caller may have changed U since the last call
    SISDC_TRY(lv->ctx, sweep(lv, u0, U, g, dt, nsweeps));
}

sisdc_status sisdc_residual(sisdc_level lv, const double* u0, const double* U, const double* g, double dt,
                            double* r) {
    if (!lv || !u0 || !U || !r || !(dt > 0.0)) return SISDC_E_ARG;
    lv->valid = false;
    SISDC_TRY(lv->ctx, residual(lv, u0, U, g, dt, r));
}

sisdc_status sisdc_transfer(sisdc_level fine, sisdc_level coarse, int op, const double* in, double* out) {
    if (!fine || !coarse || !in || !out || op < 0 || op > 3) return SISDC_E_ARG;
    if (fine->ctx != coarse->ctx || fine->index != coarse->index + 1)
        return fail(fine->ctx, SISDC_E_ARG, "transfer needs adjacent levels of one context");
    SISDC_TRY(fine->ctx, k_transfer(fine, op, in, out, 0));
}

sisdc_status sisdc_vcycle(sisdc_ctx c, const double* u0, double* U, double dt, int Nc) {
    if (!c || !u0 || !U || !(dt > 0.0) || Nc < 0) return SISDC_E_ARG;
    if (c->levels.empty()) return fail(c, SISDC_E_STATE, "no level created");
    try {
        const int nl = (int)c->levels.size();
        LevelPtrs P;
        P.u0.resize(nl);
        P.U.resize(nl);
        for (int l = 0; l < nl; ++l) {
            P.u0[l] = l == nl - 1 ? u0 : c->levels[l]->u0;
            P.U[l] = l == nl - 1 ? U : c->levels[l]->U;
            c->levels[l]->valid = false;
        }
        for (int l = nl - 1; l >= 1; --l) k_transfer(c->levels[l], T_PROJECT_SPACE, P.u0[l], c->levels[l - 1]->u0, 0);
        vcycle(c, P, nl, dt, Nc);
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_step(sisdc_ctx c, double* u, double t, double dt, int ncycles, int start, int post) {
    (void)t;
    if (!c || !u || !(dt > 0.0) || ncycles < 0 || start < 0 || start > 3) return SISDC_E_ARG;
    if (c->levels.empty()) return fail(c, SISDC_E_STATE, "no level created");
    try {
        if (!c->prob.use_graph) {
            enqueue_step(c, u, dt, ncycles, start, post);
            return SISDC_OK;
        }
        if (!(c->gexec && c->g_u == u && c->g_dt == dt && c->g_ncycles == ncycles && c->g_start == start &&
              c->g_post == post)) {
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            cudaGraph_t graph = nullptr;
            const long long l0 = c->launches;
            long long s0[8];
            for (int l = 0; l < 8; ++l) s0[l] = c->sweeps[l];
            check(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            try {
                enqueue_step(c, u, dt, ncycles, start, post);
                c->g_launches = c->launches - l0;
                c->launches = l0;
                for (int l = 0; l < 8; ++l) {
                    c->g_sweeps[l] = c->sweeps[l] - s0[l];
                    c->sweeps[l] = s0[l];
                }
            } catch (...) {
                cudaStreamEndCapture(c->stream, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            check(c, cudaStreamEndCapture(c->stream, &graph), "end capture");
            cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            check(c, e, "graph instantiate");
            c->g_u = u; c->g_dt = dt; c->g_ncycles = ncycles; c->g_start = start; c->g_post = post;
        }
        check(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch");
        c->launches += c->g_launches;
        for (int l = 0; l < 8; ++l) c->sweeps[l] += c->g_sweeps[l];
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_norms(sisdc_level lv, const double* u, const double* ref, double* l2, double* mass,
                         double* maxabs) {
    if (!lv || !u) return SISDC_E_ARG;
    sisdc_ctx_s* c = lv->ctx;
    const int nc = c->prob.ncomp;
    cudaError_t e = launch_norms(lv->geo, u, ref, c->d_norms, c->stream);
    std::vector<double> h(3 * nc);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), c->d_norms + (size_t)norms_scratch_doubles(nc) - 3 * nc, 3 * nc * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("norms: ") + cudaGetErrorString(e));
    c->launches += 2;
    for (int q = 0; q < nc; ++q) {
        if (l2) l2[q] = h[3 * q];
        if (mass) mass[q] = h[3 * q + 1];
        if (maxabs) maxabs[q] = h[3 * q + 2];
    }
    return SISDC_OK;
}

sisdc_status sisdc_sync(sisdc_ctx c) {
    if (!c) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("flag read: ") + cudaGetErrorString(e));
    if (flag) {
        cudaMemset(c->d_err, 0, sizeof(int));
        if (flag & DEV_TIMEOUT) {
            cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned));
            return fail(c, SISDC_E_TIMEOUT, "a grid barrier wait timed out");
        }
        if (flag & DEV_NONFINITE) return fail(c, SISDC_E_NONFINITE, "non-finite value in an implicit solve");
        if (flag & DEV_NOCONV) return fail(c, SISDC_E_NOCONV, "an implicit solve reached cg_maxit");
    }
    return SISDC_OK;
}

sisdc_status sisdc_get_stats(sisdc_ctx c, sisdc_stats* out) {
    if (!c || !out) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    long long s[ST_N] = {0};
    if (e == cudaSuccess) e = cudaMemcpy(s, c->d_stats, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("stats: ") + cudaGetErrorString(e));
    std::memset(out, 0, sizeof(*out));
    out->cg_solves = s[ST_SOLVES];
    out->cg_iters = s[ST_ITERS];
    out->cg_max_iters = s[ST_MAXIT];
    out->cg_noconv = s[ST_NOCONV];
    out->ir_steps = s[ST_IR];
    for (int l = 0; l < 8; ++l) out->sweeps[l] = c->sweeps[l];
    out->launches = c->launches;
    return SISDC_OK;
}

sisdc_status sisdc_reset_stats(sisdc_ctx c) {
    if (!c) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, ST_N * sizeof(long long));
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("reset: ") + cudaGetErrorString(e));
    for (int l = 0; l < 8; ++l) c->sweeps[l] = 0;
    c->launches = 0;
    return SISDC_OK;
}

sisdc_status sisdc_level_config(sisdc_level lv, int* h_epb, int* h_grid, int* h_block) {
    if (!lv) return SISDC_E_ARG;
    if (h_epb) *h_epb = lv->sw_epb;
    if (h_grid) *h_grid = lv->sw_grid;
    if (h_block) *h_block = lv->sw_block;
    return SISDC_OK;
}

// Tile-shape autotuner of the persistent sweep kernel: per level, every
// candidate (elements per tile, blocks in the grid) runs one refresh and one
// timed correction sweep from the caller's state (projected to the level,
// spread over its nodes); the fastest is kept.
sisdc_status sisdc_autotune(sisdc_ctx c, const double* d_u, double dt, int reps, int* h_config) {
    if (!c || !d_u || !(dt > 0.0) || reps < 1) return SISDC_E_ARG;
    if (c->levels.empty()) return fail(c, SISDC_E_STATE, "no level created");
    std::vector<sisdc_level_s*>& L = c->levels;
    const int nl = (int)L.size();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        check(c, cudaEventCreate(&e0), "event");
        check(c, cudaEventCreate(&e1), "event");
        copy_d2d(L[nl - 1], L[nl - 1]->u0, d_u, L[nl - 1]->NV);
        for (int l = nl - 1; l >= 1; --l) k_transfer(L[l], T_PROJECT_SPACE, L[l]->u0, L[l - 1]->u0, 0);
        for (int l = 0; l < nl; ++l) {
            sisdc_level_s* lv = L[l];
            auto spread = [&]() {
                for (int m = 0; m < lv->M; ++m) copy_d2d(lv, Um(lv, lv->U, m), lv->u0, lv->NV);
            };
            const int maxepb = lv->Q >= 512 ? 1 : 512 / lv->Q;
            std::vector<int> cand;
            for (int e : {maxepb, (3 * maxepb) / 4, maxepb / 2, maxepb / 3, maxepb / 4, lv->sw_epb, 2, 1})
                if (e >= 1 && e <= maxepb && std::find(cand.begin(), cand.end(), e) == cand.end()) cand.push_back(e);
            float best = 0.0f;
            int best_epb = lv->sw_epb, best_grid = lv->sw_grid, best_block = lv->sw_block;
            for (int e : cand) {
                int epb = e, block = 0;
                const int gmax = sweep_config(lv->geo, c->prob.pde, lv->mix ? 1 : 0, &epb, &block);
                if (gmax < 1 || gmax > c->max_grid) continue;
                // fewer blocks than tiles trade FP64 parallelism for cheaper grid
                // barriers (small, latency-bound levels)
                int last = 0;
                for (int grid : {gmax, gmax / 2, gmax / 4}) {
                    if (grid < 1 || grid == last || (grid != gmax && grid < 8)) continue;
                    last = grid;
                    lv->sw_epb = epb;
                    lv->sw_grid = grid;
                    lv->sw_block = block;
                    float t = 0.0f;
                    for (int r = 0; r < reps; ++r) {
                        spread();
                        refresh(lv, lv->u0, lv->U);
                        check(c, cudaEventRecord(e0, c->stream), "event");
                        run_sweep_kernel(lv, SW_CORRECT, lv->u0, lv->U, nullptr, dt, 1);
                        check(c, cudaEventRecord(e1, c->stream), "event");
                        check(c, cudaEventSynchronize(e1), "event sync");
                        float ms = 0.0f;
                        check(c, cudaEventElapsedTime(&ms, e0, e1), "event time");
                        t = r == 0 ? ms : std::min(t, ms);
                    }
                    if (best == 0.0f || t < best) {
                        best = t;
                        best_epb = epb;
                        best_grid = grid;
                        best_block = block;
                    }
                }
            }
            lv->sw_epb = best_epb;
            lv->sw_grid = best_grid;
            lv->sw_block = best_block;
            lv->valid = false;
            if (h_config) {
                h_config[3 * l] = best_epb;
                h_config[3 * l + 1] = best_grid;
                h_config[3 * l + 2] = best_block;
            }
        }
        check(c, cudaStreamSynchronize(c->stream), "sync");
    } catch (const Fail& f) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return f.st;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    // the timing runs count nothing
    cudaMemset(c->d_stats, 0, ST_N * sizeof(long long));
    for (int l = 0; l < 8; ++l) c->sweeps[l] = 0;
    c->launches = 0;
    return sisdc_sync(c);
}

sisdc_status sisdc_set_kernel_timing(sisdc_ctx c, int enable, int level) {
    if (!c) return SISDC_E_ARG;
    if (enable && c->prob.use_graph) return fail(c, SISDC_E_STATE, "kernel timing needs eager mode (use_graph = 0)");
    c->timing = enable != 0;
    c->timing_level = level;
    c->ev_used = 0;
    c->ev_level.clear();
    c->ev_sweeps.clear();
    return SISDC_OK;
}

sisdc_status sisdc_get_kernel_timing(sisdc_ctx c, double* ms_total, long long* launches, long long* iters,
                                     long long* nodes_x_iters, long long* dof_sweeps) {
    if (!c) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("sync: ") + cudaGetErrorString(e));
    const size_t n = c->ev_used / 2;
    std::vector<int> it(n);
    if (n) {
        e = cudaMemcpy(it.data(), c->d_iters, n * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    }
    double tot = 0.0;
    long long its = 0, nxi = 0, sweeps_nv = 0;
    for (size_t k = 0; k < n; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]);
        if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("elapsed: ") + cudaGetErrorString(e));
        tot += ms;
        its += it[k];
        nxi += (long long)it[k] * c->levels[c->ev_level[k]]->NV;
        sweeps_nv += (long long)c->ev_sweeps[k] * c->levels[c->ev_level[k]]->NV;
    }
    if (ms_total) *ms_total = tot;
    if (launches) *launches = (long long)n;
    if (iters) *iters = its;
    if (nodes_x_iters) *nodes_x_iters = nxi;
    if (dof_sweeps) *dof_sweeps = sweeps_nv;
    c->ev_used = 0;
    c->ev_level.clear();
    c->ev_sweeps.clear();
    return SISDC_OK;
}

const char* sisdc_last_error(sisdc_ctx c) { return c ? c->err.c_str() : "null context"; }

sisdc_status sisdc_set_solve_log(sisdc_ctx c, int level, double* d_r, double* d_dx, double* d_c, int capacity) {
    if (!c) return SISDC_E_ARG;
    if (d_r && (!d_dx || !d_c || capacity < 1 || level < 0 || level >= (int)c->levels.size()))
        return fail(c, SISDC_E_ARG, "solve log needs buffers, a capacity and an existing level");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemset(c->d_log_count, 0, sizeof(int));
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, cudaGetErrorString(e));
    c->log_level = d_r ? level : -1;
    c->log_r = d_r;
    c->log_dx = d_dx;
    c->log_c = d_c;
    c->log_cap = d_r ? capacity : 0;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return SISDC_OK;
}

sisdc_status sisdc_set_learned(sisdc_ctx c, int level, sisdc_mlp mlp) {
    if (!c || level < 0 || level >= (int)c->levels.size()) return SISDC_E_ARG;
    sisdc_level_s* lv = c->levels[level];
    if (mlp) {
        if (lv->mix) return fail(c, SISDC_E_ARG, "the learned sweep runs the FP64 form only");
        if (c->av_on) return fail(c, SISDC_E_ARG, "the learned sweep has no artificial viscosity");
        if (c->prob.use_graph)
            return fail(c, SISDC_E_STATE, "the learned sweep runs eagerly (use_graph = 0): it reads lambda(u0) "
                                          "on the host once per sweep");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, cudaGetErrorString(e));
    lv->learned = mlp;
    return SISDC_OK;
}

sisdc_status sisdc_get_solve_log_count(sisdc_ctx c, int* h_count) {
    if (!c || !h_count) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h_count, c->d_log_count, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, cudaGetErrorString(e));
    if (*h_count > c->log_cap) *h_count = c->log_cap;
    return SISDC_OK;
}

sisdc_status sisdc_mlp_apply(sisdc_mlp p, const double* d_r, double c, double* d_z, int add);

namespace {
double host_dot(sisdc_level_s* lv, const double* a, const double* b, int jacobi, double cval) {
    sisdc_ctx_s* c = lv->ctx;
    check(c, launch_dot(lv->geo, a, b, jacobi, cval, c->d_norms, c->stream), "dot kernel");
    double v = 0.0;
    check(c, cudaMemcpyAsync(&v, c->d_norms + 256, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    check(c, cudaStreamSynchronize(c->stream), "sync");
    c->launches += 2;
    return v;
}

// M-weighted residual M rhs - (M + cA) x
void residual_into(sisdc_level_s* lv, const double* x, const double* rhs, double cval, double* out) {
    k_lap(lv, x, out, APPLY_RES, nullptr, rhs, Coef{cval, 0.0, nullptr});
}
// nodal residual rhs - (x - c L x), the input of the learned correction
void nodal_residual_into(sisdc_level_s* lv, const double* x, const double* rhs, double cval, double* out) {
    k_lap(lv, x, out, APPLY_RESN, nullptr, rhs, Coef{cval, 0.0, nullptr});
}
}  // namespace

sisdc_status sisdc_solve_learned(sisdc_level lv, sisdc_mlp mlp, double cval, const double* rhs, double* x, int mode,
                                 int* h_iters) {
    if (!lv || !rhs || !x || !(cval > 0.0) || mode < 0 || mode > 2 || (mode > 0 && !mlp)) return SISDC_E_ARG;
    sisdc_ctx_s* c = lv->ctx;
    const long long NV = lv->NV;
    try {
        if (mode <= 1) {
            if (mode == 1) {
                nodal_residual_into(lv, x, rhs, cval, lv->cg_r);
                sisdc_status st = sisdc_mlp_apply(mlp, lv->cg_r, cval, x, 1);
                if (st != SISDC_OK) return fail(c, st, "MLP application failed");
            }
            return sisdc_solve(lv, cval, rhs, x, h_iters);
        }
        // flexible CG, MLP preconditioner (Polak-Ribiere beta), MLP initial guess
        double* R = lv->cg_r;
        double* Z = lv->dC;
        double* Pv = lv->cg_p;
        double* AP = lv->cg_Ap;
        double* Rold = lv->V;
        double* Dv = lv->V + NV;
        check(c, cudaMemsetAsync(lv->tmpc, 0, NV * sizeof(double), c->stream), "memset");
        residual_into(lv, lv->tmpc, rhs, cval, Dv);                // M b
        const double bb = host_dot(lv, Dv, Dv, 1, cval);
        const double tol2 = std::max(c->prob.cg_rtol * c->prob.cg_rtol * bb, 1e-300);
        nodal_residual_into(lv, x, rhs, cval, R);
        sisdc_status st = sisdc_mlp_apply(mlp, R, cval, x, 1);
        if (st != SISDC_OK) return fail(c, st, "MLP application failed");
        residual_into(lv, x, rhs, cval, R);
        nodal_residual_into(lv, x, rhs, cval, lv->tmpc);
        st = sisdc_mlp_apply(mlp, lv->tmpc, cval, Z, 0);
        if (st != SISDC_OK) return fail(c, st, "MLP application failed");
        copy_d2d(lv, Pv, Z, NV);
        double rz = host_dot(lv, R, Z, 0, cval);
        int it = 0;
        while (it < c->prob.cg_maxit) {
            const double rr = host_dot(lv, R, R, 1, cval);
            if (!(rr > tol2)) break;
            if (!(rz > 0.0)) {                                     // breakdown: fall back to Jacobi-PCG
                int more = 0;
                sisdc_status s2 = sisdc_solve(lv, cval, rhs, x, &more);
                if (h_iters) *h_iters = it + more;
                return s2;
            }
            k_lap(lv, Pv, AP, APPLY_OP, nullptr, nullptr, Coef{cval, 0.0, nullptr});
            const double alpha = rz / host_dot(lv, Pv, AP, 0, cval);
            Terms tx;
            tx.add(x, 1.0);
            tx.add(Pv, alpha);
            k_lin(lv, x, tx);
            copy_d2d(lv, Rold, R, NV);
            Terms tr;
            tr.add(R, 1.0);
            tr.add(AP, -alpha);
            k_lin(lv, R, tr);
            // the network's input, the nodal residual rhs - (x - c L x), is M^-1 R
            // of the recurrence residual: no operator application per iteration
            check(c, launch_minv(lv->geo, R, lv->tmpc, c->stream), "mass scaling kernel");
            c->launches++;
            st = sisdc_mlp_apply(mlp, lv->tmpc, cval, Z, 0);
            if (st != SISDC_OK) return fail(c, st, "MLP application failed");
            Terms td;
            td.add(R, 1.0);
            td.add(Rold, -1.0);
            k_lin(lv, Rold, td);                                   // r_new - r_old
            const double beta = host_dot(lv, Z, Rold, 0, cval) / rz;
            rz = host_dot(lv, R, Z, 0, cval);
            Terms tp;
            tp.add(Z, 1.0);
            tp.add(Pv, beta);
            k_lin(lv, Pv, tp);
            ++it;
        }
        if (h_iters) *h_iters = it;
        if (it >= c->prob.cg_maxit) return fail(c, SISDC_E_NOCONV, "flexible CG reached cg_maxit");
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}



}  // extern "C"

namespace sisdc {
void level_shape(sisdc_level lv, int* nc, int* nex, int* ney, int* q, double* hx, double* hy, int* dim) {
    *nc = lv->ctx->prob.ncomp;
    *nex = lv->geo.nex;
    *ney = lv->geo.ney;
    *q = lv->Q;
    *hx = lv->geo.hx;
    *hy = lv->geo.hy;
    *dim = lv->desc.dim;
}
cudaStream_t level_stream(sisdc_level lv) { return lv->ctx->stream; }
}  // namespace sisdc
