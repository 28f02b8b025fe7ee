// Host orchestration and C ABI of the batched ensemble: many independent 2D
// convection-diffusion problems on the periodic unit square, each advanced
// by its own two-level SI-MLSDC time step (Algorithm 2 with the Cascade start
// of Algorithm 3 or the predictor start), all instances of one polynomial
// degree handled by one persistent cooperative launch per sweep (ens.cuh).
//
// Instances are grouped by fine degree P; the coarse level of a group has
// degree ceil(P/2) (p-coarsening, Sec. 6.2) and the same element grids.  The
// packed state vector holds the groups in increasing P, the instances of a
// group in their input order, each as [ey][ex][node] on its own grid.  The
// space-time transfers act per element and need no instance information; the
// FAS residual kernel reads each element's time step through its instance.
// A whole ensemble step (all groups) is queued without host synchronisation
// and can be captured as one CUDA graph.
//
// Tile shapes: the elements per tile (block = tile elements x nodes per
// element threads) and the blocks per SM of each level are chosen by
// sisdc_ens_autotune, which times one correction sweep of each candidate on
// the caller's state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sisdc.h"
#include "ops.h"
#include "tables.h"

namespace sisdc {
int ens_occupancy_lo(int nq, int epb);
int ens_occupancy_hi(int nq, int epb);
int ens_occupancy_lo_mix(int nq, int epb);
int ens_occupancy_hi_mix(int nq, int epb);
cudaError_t ens_launch_lo(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_hi(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_lo_mix(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_hi_mix(const EnsArgs& a, int nq, int grid, cudaStream_t s);
int ens_occupancy_lo2(int nq, int epb);
int ens_occupancy_hi2(int nq, int epb);
int ens_occupancy_lo_mix2(int nq, int epb);
int ens_occupancy_hi_mix2(int nq, int epb);
cudaError_t ens_launch_lo2(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_hi2(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_lo_mix2(const EnsArgs& a, int nq, int grid, cudaStream_t s);
cudaError_t ens_launch_hi_mix2(const EnsArgs& a, int nq, int grid, cudaStream_t s);

int ens_occupancy(int nq, int mix, int epb) {
    if (mix) return nq < 6 ? ens_occupancy_lo_mix(nq, epb) : ens_occupancy_hi_mix(nq, epb);
    return nq < 6 ? ens_occupancy_lo(nq, epb) : ens_occupancy_hi(nq, epb);
}

// blocks per SM of the register-capped variant
int ens_occupancy_capped(int nq, int mix, int epb) {
    if (mix) return nq < 6 ? ens_occupancy_lo_mix2(nq, epb) : ens_occupancy_hi_mix2(nq, epb);
    return nq < 6 ? ens_occupancy_lo2(nq, epb) : ens_occupancy_hi2(nq, epb);
}

cudaError_t launch_ens_sweep(const EnsArgs& a, int nq, int mix, int grid, cudaStream_t s, int capped) {
    if (mix && capped) return nq < 6 ? ens_launch_lo_mix2(a, nq, grid, s) : ens_launch_hi_mix2(a, nq, grid, s);
    if (mix) return nq < 6 ? ens_launch_lo_mix(a, nq, grid, s) : ens_launch_hi_mix(a, nq, grid, s);
    if (capped) return nq < 6 ? ens_launch_lo2(a, nq, grid, s) : ens_launch_hi2(a, nq, grid, s);
    return nq < 6 ? ens_launch_lo(a, nq, grid, s) : ens_launch_hi(a, nq, grid, s);
}

// F^nn / FAS residual with per-element time steps:
// r[m] = (residual ? (g ? g[m] : 0) - fnn_m : fnn_m),
// fnn_m = U[m] - U[m-1] - dt_e sum_j W[m][j] F[j],  U[-1] = u0.
struct EnsFnnArgs {
    const double *u0, *U, *F, *g;
    double* r;
    const int* elem_inst;
    const EnsInst* inst;
    double W[MMAX * MMAX];
    int M, Q, residual;
    long long n;
};

__global__ void k_ens_fnn(const __grid_constant__ EnsFnnArgs a) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n;
         idx += (long long)gridDim.x * blockDim.x) {
        const double dt = a.inst[a.elem_inst[idx / a.Q]].dt;
        double f[MMAX];
        for (int i = 0; i < a.M; ++i) f[i] = a.F[i * a.n + idx];
        double prev = a.u0[idx];
        for (int m = 0; m < a.M; ++m) {
            double s = 0.0;
            for (int i = 0; i < a.M; ++i) s += a.W[m * a.M + i] * f[i];
            const double cur = a.U[m * a.n + idx];
            const double fnn = cur - prev - dt * s;
            a.r[m * a.n + idx] = a.residual ? ((a.g ? a.g[m * a.n + idx] : 0.0) - fnn) : fnn;
            prev = cur;
        }
    }
}

}  // namespace sisdc

using namespace sisdc;

namespace {

struct EnsLevel {
    int P = 0, nq = 0, Q = 0, M = 0;
    bool mix = false;
    long long nel = 0, N = 0;
    LevelTables tab;
    std::vector<EnsInst> hinst;
    double* d_tab = nullptr;        // D, K, w, dl, then the transfer tables of a fine level
    EnsInst* d_inst = nullptr;
    int* d_elem_inst = nullptr;
    double* d_mem = nullptr;
    double *U = nullptr, *F = nullptr, *CC = nullptr, *LU = nullptr, *Qb = nullptr, *G = nullptr, *V = nullptr,
           *R = nullptr, *u0 = nullptr, *c0 = nullptr, *dC = nullptr, *tmpc = nullptr;
    double *d_Ix = nullptr, *d_Px = nullptr, *d_Rx = nullptr, *d_It = nullptr, *d_Pt = nullptr, *d_Rt = nullptr,
           *d_one = nullptr;
    // launch configuration
    int epb = 0, grid = 0, lmax = 0;
    int capped = 0;             // 1: the register-capped kernel (more blocks per SM than the plain one holds)
    long long ntiles = 0;
    int4* d_tiles = nullptr;
    int* d_nloc = nullptr;
    int* d_loc_inst = nullptr;
    bool valid = false;
};

struct EnsGroup {
    int P = 0;
    int index = 0;                // position in the ensemble's group list
    std::vector<int> members;     // instance indices
    long long off = 0;            // offset of the group in the packed state
    EnsLevel lv[2];               // 0 = coarse, 1 = fine
};

}  // namespace

struct sisdc_ens_s {
    sisdc_ens_opts opts{};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    int nsm = 0;
    std::vector<sisdc_ens_instance> inst;
    std::vector<EnsGroup*> groups;
    std::vector<long long> offset;     // [n + 1]
    std::vector<int> group_of, index_in_group;
    long long total = 0;
    long long maxN = 0;
    long long maxT = 0;                 // largest level's face-trace array (doubles)
    // shared scratch (launches are serialised on the stream)
    double *cg_r = nullptr, *cg_p = nullptr, *cg_p2 = nullptr, *cg_Ap = nullptr, *cg_rf = nullptr;
    double *cg_tz = nullptr, *cg_tp0 = nullptr, *cg_tp1 = nullptr;   // FP64 CG face traces
    double* part = nullptr;
    size_t part_cap = 0;
    void* loc = nullptr;
    size_t loc_cap = 0;
    double* loc_dinv = nullptr;
    size_t dinv_cap = 0;
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    long long* d_stats = nullptr;
    long long* d_inst_iters = nullptr;   // [n], indexed through the groups
    std::vector<long long*> iters_view;   // per group level: d_inst_iters slice (fine level only)
    long long launches = 0;
    long long sweeps[2] = {0, 0};
    std::string err;
    // measurement hook: events around fine-level correction launches, per group
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_group;
    size_t ev_used = 0;
    cudaGraphExec_t gexec = nullptr;
    double* g_u = nullptr;
    long long g_launches = 0, g_sweeps[2] = {0, 0};   // per replay of the captured step
};

namespace {

struct Fail {
    sisdc_status st;
};

void check(sisdc_ens_s* c, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{e == cudaErrorMemoryAllocation ? SISDC_E_OOM : SISDC_E_CUDA};
    }
}

sisdc_status fail(sisdc_ens_s* c, sisdc_status st, const std::string& msg) {
    c->err = msg;
    return st;
}

template <class T>
void dmalloc(sisdc_ens_s* c, T** p, size_t n) {
    check(c, cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)), "allocation");
}

void release_level(EnsLevel& L) {
    cudaFree(L.d_tab);
    cudaFree(L.d_inst);
    cudaFree(L.d_elem_inst);
    cudaFree(L.d_mem);
    cudaFree(L.d_tiles);
    cudaFree(L.d_nloc);
    cudaFree(L.d_loc_inst);
    L = EnsLevel();
}

// geometry record of one instance on a level of degree P
EnsInst make_inst(const sisdc_ens_instance& s, int nq, const LevelTables& tab, long long e0) {
    EnsInst I{};
    I.e0 = e0;
    I.nex = s.nel[0];
    I.ney = s.nel[1];
    I.hx = 1.0 / s.nel[0];
    I.hy = 1.0 / s.nel[1];
    I.sx = 2.0 / I.hx;
    I.sy = 2.0 / I.hy;
    I.ihx = 1.0 / I.hx;
    I.ihy = 1.0 / I.hy;
    I.taux = 2.0 * nq * nq / I.hx;
    I.tauy = 2.0 * nq * nq / I.hy;
    I.liftLx = I.sx / tab.w[0];
    I.liftRx = I.sx / tab.w[nq - 1];
    I.liftLy = I.sy / tab.w[0];
    I.liftRy = I.sy / tab.w[nq - 1];
    I.ax = s.adv[0];
    I.ay = s.adv[1];
    I.nu = s.nu;
    I.lam = std::max(std::fabs(s.adv[0]), std::fabs(s.adv[1]));
    I.dt = s.dt;
    I.rho = I.hy / I.hx;
    I.irho = I.hx / I.hy;
    I.mq = 0.25 * I.hx * I.hy;
    I.imq = 1.0 / I.mq;
    return I;
}

void build_level(sisdc_ens_s* c, EnsGroup& g, int which, int P, int M, bool fine) {
    EnsLevel& L = g.lv[which];
    L.P = P;
    L.nq = P + 1;
    L.Q = L.nq * L.nq;
    L.M = M;
    const int ml = c->opts.mixed_levels;
    L.mix = c->opts.precision == SISDC_MIXED && P >= 3 && (ml == 0 || ((ml >> (fine ? 1 : 0)) & 1));
    if (!build_level_tables(P, M, c->opts.nodes == SISDC_LOBATTO, &L.tab)) {
        c->err = "table construction failed";
        throw Fail{SISDC_E_ARG};
    }
    const int nq = L.nq;
    std::vector<double> tab(2 * nq * nq + 2 * nq);
    for (int k = 0; k < nq * nq; ++k) {
        tab[k] = L.tab.D[k];
        tab[nq * nq + k] = L.tab.K[k];
    }
    for (int i = 0; i < nq; ++i) {
        tab[2 * nq * nq + i] = L.tab.w[i];
        // h * (diagonal of the 1D SIPG line operator): 2 K_ii plus the face
        // terms of the end nodes, with the penalty h tau = 2 (P+1)^2
        double d = 2.0 * L.tab.Kdiag[i];
        if (i == nq - 1) d += -2.0 * L.tab.DPP + 2.0 * nq * nq;
        if (i == 0) d += 2.0 * L.tab.D00 + 2.0 * nq * nq;
        tab[2 * nq * nq + nq + i] = d;
    }
    if (fine) {
        const EnsLevel& C = g.lv[0];
        std::vector<double> Ix = lagrange_matrix(C.tab.gll, L.tab.gll);
        std::vector<double> Px = lagrange_matrix(L.tab.gll, C.tab.gll);
        std::vector<double> Rx(C.nq * nq);
        for (int a = 0; a < C.nq; ++a)
            for (int b = 0; b < nq; ++b) Rx[a * nq + b] = Ix[b * C.nq + a] * L.tab.w[b] / C.tab.w[a];
        std::vector<double> It = lagrange_matrix(C.tab.tau, L.tab.tau);
        std::vector<double> Pt = lagrange_matrix(L.tab.tau, C.tab.tau);
        std::vector<double> Rt(C.M * M);
        for (int a = 0; a < C.M; ++a)
            for (int b = 0; b < M; ++b) Rt[a * M + b] = It[b * C.M + a];
        for (const std::vector<double>* v : {&Ix, &Px, &Rx, &It, &Pt, &Rt}) tab.insert(tab.end(), v->begin(), v->end());
        tab.push_back(1.0);
        const size_t base = 2 * nq * nq + 2 * nq;
        dmalloc(c, &L.d_tab, tab.size());
        L.d_Ix = L.d_tab + base;
        L.d_Px = L.d_Ix + Ix.size();
        L.d_Rx = L.d_Px + Px.size();
        L.d_It = L.d_Rx + Rx.size();
        L.d_Pt = L.d_It + It.size();
        L.d_Rt = L.d_Pt + Pt.size();
        L.d_one = L.d_Rt + Rt.size();
    } else {
        dmalloc(c, &L.d_tab, tab.size());
    }
    check(c, cudaMemcpy(L.d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice), "table upload");
    // instances and the element -> instance map
    std::vector<int> elem_inst;
    long long e0 = 0;
    for (size_t k = 0; k < g.members.size(); ++k) {
        const sisdc_ens_instance& s = c->inst[g.members[k]];
        L.hinst.push_back(make_inst(s, nq, L.tab, e0));
        const long long ne = (long long)s.nel[0] * s.nel[1];
        elem_inst.insert(elem_inst.end(), (size_t)ne, (int)k);
        e0 += ne;
    }
    L.nel = e0;
    L.N = e0 * L.Q;
    dmalloc(c, &L.d_inst, L.hinst.size());
    dmalloc(c, &L.d_elem_inst, elem_inst.size());
    check(c, cudaMemcpy(L.d_elem_inst, elem_inst.data(), elem_inst.size() * sizeof(int), cudaMemcpyHostToDevice),
          "map upload");
    const long long N = L.N, MV = (long long)M * N;
    const long long total = 8 * MV + 4 * N;
    dmalloc(c, &L.d_mem, total);
    check(c, cudaMemset(L.d_mem, 0, total * sizeof(double)), "memset");
    double* p = L.d_mem;
    auto take = [&](long long n) { double* q = p; p += n; return q; };
    L.U = take(MV); L.F = take(MV); L.CC = take(MV); L.LU = take(MV);
    L.Qb = take(MV); L.G = take(MV); L.V = take(MV); L.R = take(MV);
    L.u0 = take(N); L.c0 = take(N); L.dC = take(N); L.tmpc = take(N);
    c->maxN = std::max(c->maxN, N);
    c->maxT = std::max(c->maxT, L.nel * 8LL * L.nq);
}

// Tiles of epb elements per instance (never straddling two), owned
// round-robin by `grid` blocks; per block the list of instances it touches.
void configure(sisdc_ens_s* c, EnsLevel& L, int epb, int grid) {
    std::vector<int4> tiles;
    for (size_t k = 0; k < L.hinst.size(); ++k) {
        EnsInst& I = L.hinst[k];
        const long long ne = (long long)I.nex * I.ney;
        I.t0 = (int)tiles.size();
        for (long long e = 0; e < ne; e += epb)
            tiles.push_back(make_int4((int)k, 0, (int)(I.e0 + e), (int)std::min<long long>(epb, ne - e)));
        I.nt = (int)tiles.size() - I.t0;
    }
    const long long nt = (long long)tiles.size();
    if (grid > nt) grid = (int)nt;
    std::vector<std::vector<int>> loc(grid);
    for (long long t = 0; t < nt; ++t) {
        std::vector<int>& l = loc[t % grid];
        if (l.empty() || l.back() != tiles[t].x) l.push_back(tiles[t].x);
        tiles[t].y = (int)l.size() - 1;
    }
    int lmax = 1;
    for (auto& l : loc) lmax = std::max(lmax, (int)l.size());
    std::vector<int> nloc(grid), loc_inst((size_t)grid * lmax, -1);
    for (int b = 0; b < grid; ++b) {
        nloc[b] = (int)loc[b].size();
        for (size_t k = 0; k < loc[b].size(); ++k) loc_inst[(size_t)b * lmax + k] = loc[b][k];
    }
    cudaFree(L.d_tiles);
    cudaFree(L.d_nloc);
    cudaFree(L.d_loc_inst);
    L.d_tiles = nullptr;
    L.d_nloc = nullptr;
    L.d_loc_inst = nullptr;
    dmalloc(c, &L.d_tiles, tiles.size());
    dmalloc(c, &L.d_nloc, nloc.size());
    dmalloc(c, &L.d_loc_inst, loc_inst.size());
    check(c, cudaMemcpy(L.d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
    check(c, cudaMemcpy(L.d_nloc, nloc.data(), nloc.size() * sizeof(int), cudaMemcpyHostToDevice), "upload");
    check(c, cudaMemcpy(L.d_loc_inst, loc_inst.data(), loc_inst.size() * sizeof(int), cudaMemcpyHostToDevice), "upload");
    check(c, cudaMemcpy(L.d_inst, L.hinst.data(), L.hinst.size() * sizeof(EnsInst), cudaMemcpyHostToDevice), "upload");
    L.epb = epb;
    L.grid = grid;
    L.lmax = lmax;
    // more co-resident blocks than the plain kernel holds: the register-capped one
    L.capped = grid > ens_occupancy(L.nq, L.mix ? 1 : 0, epb) * c->nsm ? 1 : 0;
    L.ntiles = nt;
    // shared scratch large enough for this configuration
    const size_t np = (size_t)(2 * 4 * L.hinst.size() + 2) * grid;
    if (np > c->part_cap) {
        cudaFree(c->part);
        c->part = nullptr;
        dmalloc(c, &c->part, np);
        c->part_cap = np;
    }
    const size_t nl = (size_t)grid * lmax * 128;   // bytes; EnsLocal is smaller
    if (nl > c->loc_cap) {
        cudaFree(c->loc);
        c->loc = nullptr;
        check(c, cudaMalloc(&c->loc, nl), "allocation");
        c->loc_cap = nl;
    }
    const size_t nd = (size_t)grid * lmax * L.Q;
    if (nd > c->dinv_cap) {
        cudaFree(c->loc_dinv);
        c->loc_dinv = nullptr;
        dmalloc(c, &c->loc_dinv, nd + (nd + 1) / 2);         // FP64 factors, then their FP32 copy
        c->dinv_cap = nd;
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
}

// default shape: the largest tile (at most 512 threads), all co-resident blocks
void configure_default(sisdc_ens_s* c, EnsLevel& L) {
    int epb = std::max(1, 512 / L.Q);
    int per = ens_occupancy(L.nq, L.mix ? 1 : 0, epb);
    while (per < 1 && epb > 1) per = ens_occupancy(L.nq, L.mix ? 1 : 0, --epb);
    if (per < 1) {
        c->err = "ensemble kernel cannot be launched for this degree";
        throw Fail{SISDC_E_CUDA};
    }
    configure(c, L, epb, per * c->nsm);
}

// ---- queued operations ---------------------------------------------------------
void run_sweep(sisdc_ens_s* c, EnsGroup& g, int which, int mode, const double* G, int nsweeps) {
    EnsLevel& L = g.lv[which];
    EnsArgs a{};
    a.inst = L.d_inst;
    a.ninst = (int)L.hinst.size();
    a.tiles = L.d_tiles;
    a.ntiles = L.ntiles;
    a.epb = L.epb;
    a.nloc = L.d_nloc;
    a.loc_inst = L.d_loc_inst;
    a.lmax = L.lmax;
    a.loc = c->loc;
    a.loc_dinv = c->loc_dinv;
    a.loc_dinv32 = reinterpret_cast<float*>(c->loc_dinv + c->dinv_cap);
    a.N = L.N;
    a.D = L.d_tab;
    a.K = L.d_tab + L.nq * L.nq;
    a.w = L.d_tab + 2 * L.nq * L.nq;
    a.dl = a.w + L.nq;
    a.mode = mode;
    a.nsweeps = nsweeps;
    a.stages = c->opts.si_stages;
    a.M = L.M;
    for (int m = 0; m < L.M; ++m) a.dtau[m] = L.tab.dtau[m];
    for (int k = 0; k < L.M * L.M; ++k) a.W[k] = L.tab.wnn[k];
    a.u0 = L.u0;
    a.U = L.U;
    a.G = G;
    a.F = L.F; a.CC = L.CC; a.LU = L.LU; a.Qb = L.Qb; a.c0 = L.c0; a.dC = L.dC; a.tmpc = L.tmpc;
    a.r = c->cg_r; a.p = c->cg_p; a.p2 = c->cg_p2; a.Ap = c->cg_Ap; a.rf = c->cg_rf;
    a.tz = c->cg_tz; a.tp0 = c->cg_tp0; a.tp1 = c->cg_tp1;
    a.part = c->part;
    a.bar_count = c->d_bar;
    a.bar_exit = c->d_bar + 1;
    a.err = c->d_err;
    a.stats = c->d_stats;
    a.rtol = c->opts.cg_rtol;
    a.maxit = c->opts.cg_maxit;
    a.inst_iters = which == 1 ? c->iters_view[g.index] : nullptr;   // fine-level counters per instance
    const bool timed = c->timing && which == 1 && mode == SW_CORRECT;
    if (timed) {
        while (c->ev.size() < c->ev_used + 2) {
            cudaEvent_t e;
            check(c, cudaEventCreate(&e), "timing event");
            c->ev.push_back(e);
        }
        check(c, cudaEventRecord(c->ev[c->ev_used], c->stream), "timing event");
    }
    check(c, launch_ens_sweep(a, L.nq, L.mix ? 1 : 0, L.grid, c->stream, L.capped), "ensemble sweep kernel");
    if (timed) {
        check(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream), "timing event");
        c->ev_used += 2;
        c->ev_group.push_back(g.index);
    }
    c->launches++;
    if (mode != SW_REFRESH) c->sweeps[which] += mode == SW_PREDICT ? 1 : nsweeps;
}

void refresh(sisdc_ens_s* c, EnsGroup& g, int which) {
    run_sweep(c, g, which, SW_REFRESH, nullptr, 0);
    g.lv[which].valid = true;
}

void sweep(sisdc_ens_s* c, EnsGroup& g, int which, const double* G, int nsweeps) {
    if (!g.lv[which].valid) refresh(c, g, which);
    if (nsweeps > 0) run_sweep(c, g, which, SW_CORRECT, G, nsweeps);
    g.lv[which].valid = true;
}

void predict(sisdc_ens_s* c, EnsGroup& g, int which) {
    run_sweep(c, g, which, SW_PREDICT, nullptr, 0);
    g.lv[which].valid = true;
}

void fnn(sisdc_ens_s* c, EnsLevel& L, const double* Gin, double* r, int residual) {
    EnsFnnArgs a{};
    a.u0 = L.u0;
    a.U = L.U;
    a.F = L.F;
    a.g = Gin;
    a.r = r;
    a.elem_inst = L.d_elem_inst;
    a.inst = L.d_inst;
    for (int k = 0; k < L.M * L.M; ++k) a.W[k] = L.tab.wnn[k];
    a.M = L.M;
    a.Q = L.Q;
    a.residual = residual;
    a.n = L.N;
    long long nb = (L.N + 255) / 256;
    nb = std::min<long long>(std::max<long long>(nb, 1), 32LL * c->nsm);
    k_ens_fnn<<<(unsigned)nb, 256, 0, c->stream>>>(a);
    check(c, cudaGetLastError(), "fnn kernel");
    c->launches++;
}

enum { T_INTERP = 0, T_PROJECT = 1, T_RESTRICT = 2, T_PROJECT_SPACE = 3 };
void transfer(sisdc_ens_s* c, EnsGroup& g, int op, const double* in, double* out, int add) {
    const EnsLevel& F = g.lv[1];
    const EnsLevel& C = g.lv[0];
    TransferArgs a{};
    a.dim = 2;
    a.ncomp = 1;
    a.nel = (int)F.nel;
    a.in = in;
    a.out = out;
    a.add = add;
    switch (op) {
        case T_INTERP: a.nqi = C.nq; a.nqo = F.nq; a.Mi = C.M; a.Mo = F.M; a.S = F.d_Ix; a.Tt = F.d_It; break;
        case T_PROJECT: a.nqi = F.nq; a.nqo = C.nq; a.Mi = F.M; a.Mo = C.M; a.S = F.d_Px; a.Tt = F.d_Pt; break;
        case T_RESTRICT: a.nqi = F.nq; a.nqo = C.nq; a.Mi = F.M; a.Mo = C.M; a.S = F.d_Rx; a.Tt = F.d_Rt; break;
        default: a.nqi = F.nq; a.nqo = C.nq; a.Mi = 1; a.Mo = 1; a.S = F.d_Px; a.Tt = F.d_one; break;
    }
    check(c, launch_transfer(a, c->stream), "transfer kernel");
    c->launches++;
}

void copy_d2d(sisdc_ens_s* c, double* dst, const double* src, long long n) {
    check(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "device copy");
}

// one two-level SI-MLSDC step of every instance of the group (Algorithm 2;
// the same sequence as the single-problem library)
void enqueue_group_step(sisdc_ens_s* c, EnsGroup& g, double* u) {
    EnsLevel& F = g.lv[1];
    EnsLevel& C = g.lv[0];
    const sisdc_ens_opts& o = c->opts;
    copy_d2d(c, F.u0, u + g.off, F.N);
    F.valid = C.valid = false;
    transfer(c, g, T_PROJECT_SPACE, F.u0, C.u0, 0);
    if (o.start == SISDC_START_PREDICTOR) {
        predict(c, g, 0);
        predict(c, g, 1);
    } else {
        predict(c, g, 0);
        sweep(c, g, 0, nullptr, 1);
        transfer(c, g, T_INTERP, C.U, F.U, 0);
        F.valid = false;
    }
    for (int k = 0; k < o.ncycles; ++k) {
        sweep(c, g, 1, nullptr, 1);                                  // fine pre-sweep
        fnn(c, F, nullptr, F.R, 1);                                  // r = -F^nn(u)
        transfer(c, g, T_PROJECT, F.U, C.U, 0);                      // v = P u
        copy_d2d(c, C.V, C.U, (long long)C.M * C.N);
        refresh(c, g, 0);
        fnn(c, C, nullptr, C.G, 0);                                  // g = F^nn(v)
        transfer(c, g, T_RESTRICT, F.R, C.G, 1);                     //   + R r
        sweep(c, g, 0, C.G, o.Nc);                                   // coarse sweeps
        LinArgs d{};
        d.n = (long long)C.M * C.N;
        d.nterms = 2;
        d.in[0] = C.U;
        d.coef[0] = Coef{1.0, 0.0, nullptr};
        d.in[1] = C.V;
        d.coef[1] = Coef{-1.0, 0.0, nullptr};
        d.out = C.R;
        check(c, launch_lincomb(d, c->stream), "lincomb kernel");
        c->launches++;
        transfer(c, g, T_INTERP, C.R, F.U, 1);                       // u += I (u_c - v)
        F.valid = false;
    }
    if (o.post_sweep) sweep(c, g, 1, nullptr, 1);
    copy_d2d(c, u + g.off, F.U + (long long)(F.M - 1) * F.N, F.N);
}

void enqueue_step(sisdc_ens_s* c, double* u) {
    for (EnsGroup* g : c->groups) enqueue_group_step(c, *g, u);
}

void destroy_all(sisdc_ens_s* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    for (EnsGroup* g : c->groups) {
        release_level(g->lv[0]);
        release_level(g->lv[1]);
        delete g;
    }
    c->groups.clear();
    cudaFree(c->cg_r);
    cudaFree(c->cg_p);
    cudaFree(c->cg_p2);
    cudaFree(c->cg_Ap);
    cudaFree(c->cg_rf);
    cudaFree(c->cg_tz);
    cudaFree(c->cg_tp0);
    cudaFree(c->cg_tp1);
    cudaFree(c->part);
    cudaFree(c->loc);
    cudaFree(c->loc_dinv);
    cudaFree(c->d_bar);
    cudaFree(c->d_err);
    cudaFree(c->d_stats);
    cudaFree(c->d_inst_iters);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
}

}  // namespace

// ============================================================================
extern "C" {

sisdc_status sisdc_ens_create(const sisdc_ens_instance* inst, int n, const sisdc_ens_opts* o, void* cuda_stream,
                              sisdc_ens* out) {
    if (!inst || n < 1 || !o || !out) return SISDC_E_ARG;
    *out = nullptr;
    if (o->M < 1 || o->M > MMAX || o->Mc < 1 || o->Mc > o->M) return SISDC_E_ARG;
    if (o->nodes != SISDC_RADAU_RIGHT && o->nodes != SISDC_LOBATTO) return SISDC_E_ARG;
    if (o->nodes == SISDC_LOBATTO && o->Mc < 2) return SISDC_E_ARG;
    if (o->precision != SISDC_FP64 && o->precision != SISDC_MIXED) return SISDC_E_ARG;
    if (o->mixed_levels < 0 || o->mixed_levels > 3) return SISDC_E_ARG;
    if (o->si_stages != 1 && o->si_stages != 2) return SISDC_E_ARG;
    if (!(o->cg_rtol > 0.0) || o->cg_maxit < 1 || o->Nc < 0 || o->ncycles < 0) return SISDC_E_ARG;
    if (o->start != SISDC_START_CASCADE && o->start != SISDC_START_PREDICTOR) return SISDC_E_ARG;
    for (int k = 0; k < n; ++k) {
        const sisdc_ens_instance& s = inst[k];
        if (s.P < 2 || s.P > 8 || s.nel[0] < 1 || s.nel[1] < 1 || !(s.nu >= 0.0) || !(s.dt > 0.0) ||
            !std::isfinite(s.adv[0]) || !std::isfinite(s.adv[1]))
            return SISDC_E_ARG;
        if ((long long)s.nel[0] * s.nel[1] > (1LL << 24)) return SISDC_E_ARG;
    }
    sisdc_ens_s* c = new sisdc_ens_s();
    c->opts = *o;
    c->stream = (cudaStream_t)cuda_stream;
    c->inst.assign(inst, inst + n);
    try {
        int dev = 0;
        check(c, cudaGetDevice(&dev), "device");
        check(c, cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev), "device");
        if (o->use_graph && cuda_stream == nullptr) {
            check(c, cudaStreamCreate(&c->own_stream), "stream");
            c->stream = c->own_stream;
        }
        dmalloc(c, &c->d_bar, 2);
        dmalloc(c, &c->d_err, 1);
        dmalloc(c, &c->d_stats, ST_N);
        dmalloc(c, &c->d_inst_iters, n);
        check(c, cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned)), "memset");
        check(c, cudaMemset(c->d_err, 0, sizeof(int)), "memset");
        check(c, cudaMemset(c->d_stats, 0, ST_N * sizeof(long long)), "memset");
        check(c, cudaMemset(c->d_inst_iters, 0, n * sizeof(long long)), "memset");
        // groups by fine degree, packed in increasing P
        c->group_of.assign(n, -1);
        c->index_in_group.assign(n, -1);
        for (int P = 2; P <= 8; ++P) {
            EnsGroup* g = nullptr;
            for (int k = 0; k < n; ++k) {
                if (inst[k].P != P) continue;
                if (!g) {
                    g = new EnsGroup();
                    g->P = P;
                    g->index = (int)c->groups.size();
                    c->groups.push_back(g);
                }
                c->group_of[k] = (int)c->groups.size() - 1;
                c->index_in_group[k] = (int)g->members.size();
                g->members.push_back(k);
            }
        }
        c->offset.assign(n + 1, 0);
        long long off = 0, ioff = 0;
        for (EnsGroup* g : c->groups) {
            g->off = off;
            build_level(c, *g, 0, (g->P + 1) / 2, o->Mc, false);
            build_level(c, *g, 1, g->P, o->M, true);
            for (size_t k = 0; k < g->members.size(); ++k) {
                const int i = g->members[k];
                c->offset[i] = off + g->lv[1].hinst[k].e0 * g->lv[1].Q;
            }
            off += g->lv[1].N;
            c->iters_view.push_back(c->d_inst_iters + ioff);
            ioff += (long long)g->members.size();
        }
        c->offset[n] = off;
        c->total = off;
        for (EnsGroup* g : c->groups) {
            configure_default(c, g->lv[0]);
            configure_default(c, g->lv[1]);
        }
        dmalloc(c, &c->cg_r, c->maxN);
        dmalloc(c, &c->cg_p, c->maxN);
        dmalloc(c, &c->cg_p2, c->maxN);
        dmalloc(c, &c->cg_Ap, c->maxN);
        dmalloc(c, &c->cg_rf, c->maxN);
        dmalloc(c, &c->cg_tz, c->maxT);
        dmalloc(c, &c->cg_tp0, c->maxT);
        dmalloc(c, &c->cg_tp1, c->maxT);
    } catch (const Fail& f) {
        destroy_all(c);
        delete c;
        return f.st;
    }
    *out = c;
    return SISDC_OK;
}

void sisdc_ens_destroy(sisdc_ens c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    destroy_all(c);
    delete c;
}

sisdc_status sisdc_ens_layout(sisdc_ens c, long long* offsets, long long* total) {
    if (!c) return SISDC_E_ARG;
    if (offsets)
        for (size_t k = 0; k < c->inst.size(); ++k) offsets[k] = c->offset[k];
    if (total) *total = c->total;
    return SISDC_OK;
}

sisdc_status sisdc_ens_coords(sisdc_ens c, double* hx, double* hy) {
    if (!c || !hx) return SISDC_E_ARG;
    for (size_t k = 0; k < c->inst.size(); ++k) {
        const EnsGroup* g = c->groups[c->group_of[k]];
        const EnsLevel& F = g->lv[1];
        const sisdc_ens_instance& d = c->inst[k];
        const double h0 = 1.0 / d.nel[0], h1 = 1.0 / d.nel[1];
        long long id = c->offset[k];
        for (int ey = 0; ey < d.nel[1]; ++ey)
            for (int ex = 0; ex < d.nel[0]; ++ex)
                for (int j = 0; j < F.nq; ++j)
                    for (int i = 0; i < F.nq; ++i, ++id) {
                        hx[id] = (ex + (F.tab.gll[i] + 1.0) / 2.0) * h0;
                        if (hy) hy[id] = (ey + (F.tab.gll[j] + 1.0) / 2.0) * h1;
                    }
    }
    return SISDC_OK;
}

sisdc_status sisdc_ens_set_kernel_timing(sisdc_ens c, int enable) {
    if (!c) return SISDC_E_ARG;
    if (enable && c->opts.use_graph) return fail(c, SISDC_E_STATE, "kernel timing needs eager mode (use_graph = 0)");
    c->timing = enable != 0;
    c->ev_used = 0;
    c->ev_group.clear();
    return SISDC_OK;
}

sisdc_status sisdc_ens_get_kernel_timing(sisdc_ens c, double* ms, long long* launches) {
    if (!c) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("sync: ") + cudaGetErrorString(e));
    const size_t ng = c->groups.size();
    std::vector<double> tot(ng, 0.0);
    std::vector<long long> cnt(ng, 0);
    for (size_t k = 0; k < c->ev_used / 2; ++k) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, c->ev[2 * k], c->ev[2 * k + 1]);
        if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("elapsed: ") + cudaGetErrorString(e));
        tot[c->ev_group[k]] += t;
        cnt[c->ev_group[k]] += 1;
    }
    for (size_t gi = 0; gi < ng; ++gi) {
        if (ms) ms[gi] = tot[gi];
        if (launches) launches[gi] = cnt[gi];
    }
    c->ev_used = 0;
    c->ev_group.clear();
    return SISDC_OK;
}

sisdc_status sisdc_ens_step(sisdc_ens c, double* u, int nsteps) {
    if (!c || !u || nsteps < 0) return SISDC_E_ARG;
    try {
        for (int s = 0; s < nsteps; ++s) {
            if (!c->opts.use_graph) {
                enqueue_step(c, u);
                continue;
            }
            if (!(c->gexec && c->g_u == u)) {
                if (c->gexec) {
                    cudaGraphExecDestroy(c->gexec);
                    c->gexec = nullptr;
                }
                cudaGraph_t graph = nullptr;
                const long long l0 = c->launches, s0 = c->sweeps[0], s1 = c->sweeps[1];
                check(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                try {
                    enqueue_step(c, u);
                    c->g_launches = c->launches - l0;
                    c->g_sweeps[0] = c->sweeps[0] - s0;
                    c->g_sweeps[1] = c->sweeps[1] - s1;
                    c->launches = l0;
                    c->sweeps[0] = s0;
                    c->sweeps[1] = s1;
                } catch (...) {
                    cudaStreamEndCapture(c->stream, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                check(c, cudaStreamEndCapture(c->stream, &graph), "end capture");
                cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
                cudaGraphDestroy(graph);
                check(c, e, "graph instantiate");
                c->g_u = u;
            }
            check(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch");
            c->launches += c->g_launches;
            c->sweeps[0] += c->g_sweeps[0];
            c->sweeps[1] += c->g_sweeps[1];
        }
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

sisdc_status sisdc_ens_sync(sisdc_ens c) {
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

sisdc_status sisdc_ens_get_stats(sisdc_ens c, sisdc_stats* out, long long* inst_iters) {
    if (!c || !out) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    long long s[ST_N] = {0};
    if (e == cudaSuccess) e = cudaMemcpy(s, c->d_stats, sizeof(s), cudaMemcpyDeviceToHost);
    std::vector<long long> it(c->inst.size());
    if (e == cudaSuccess && inst_iters)
        e = cudaMemcpy(it.data(), c->d_inst_iters, it.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("stats: ") + cudaGetErrorString(e));
    std::memset(out, 0, sizeof(*out));
    out->cg_solves = s[ST_SOLVES];
    out->cg_iters = s[ST_ITERS];
    out->cg_max_iters = s[ST_MAXIT];
    out->cg_noconv = s[ST_NOCONV];
    out->ir_steps = s[ST_IR];
    out->sweeps[0] = c->sweeps[0];
    out->sweeps[1] = c->sweeps[1];
    out->launches = c->launches;
    if (inst_iters)
        for (size_t k = 0; k < c->inst.size(); ++k) {
            const EnsGroup* g = c->groups[c->group_of[k]];
            inst_iters[k] = it[(c->iters_view[g->index] - c->d_inst_iters) + c->index_in_group[k]];
        }
    return SISDC_OK;
}

sisdc_status sisdc_ens_reset_stats(sisdc_ens c) {
    if (!c) return SISDC_E_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, ST_N * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_inst_iters, 0, c->inst.size() * sizeof(long long));
    if (e != cudaSuccess) return fail(c, SISDC_E_CUDA, std::string("reset: ") + cudaGetErrorString(e));
    c->sweeps[0] = c->sweeps[1] = 0;
    c->launches = 0;
    return SISDC_OK;
}

sisdc_status sisdc_ens_autotune(sisdc_ens c, const double* u, int nsweeps, int* h_config) {
    if (!c || !u || nsweeps < 1) return SISDC_E_ARG;
    try {
        cudaEvent_t e0, e1;
        check(c, cudaEventCreate(&e0), "event");
        check(c, cudaEventCreate(&e1), "event");
        for (EnsGroup* g : c->groups) {
            // a consistent state on both levels: u0 from the caller, U spread
            EnsLevel& F = g->lv[1];
            EnsLevel& C = g->lv[0];
            copy_d2d(c, F.u0, u + g->off, F.N);
            transfer(c, *g, T_PROJECT_SPACE, F.u0, C.u0, 0);
            for (int which = 0; which < 2; ++which) {
                EnsLevel& L = g->lv[which];
                for (int m = 0; m < L.M; ++m) copy_d2d(c, L.U + (long long)m * L.N, L.u0, L.N);
                std::vector<std::pair<int, int>> cand;
                const int emax = std::max(1, 512 / L.Q);
                for (int epb = emax; epb >= 1; epb = epb > 1 ? epb / 2 : 0) {
                    if (epb * L.Q < 32 && epb != emax) break;
                    const int per = std::max(ens_occupancy(L.nq, L.mix ? 1 : 0, epb),
                                             ens_occupancy_capped(L.nq, L.mix ? 1 : 0, epb));
                    for (int b = 1; b <= per; b *= 2) cand.push_back({epb, b * c->nsm});
                    if (epb == 1) break;
                }
                float best = 0.0f;
                std::pair<int, int> pick{0, 0};
                for (const auto& cf : cand) {
                    configure(c, L, cf.first, cf.second);
                    refresh(c, *g, which);
                    check(c, cudaEventRecord(e0, c->stream), "event");
                    run_sweep(c, *g, which, SW_CORRECT, nullptr, nsweeps);
                    check(c, cudaEventRecord(e1, c->stream), "event");
                    check(c, cudaEventSynchronize(e1), "event sync");
                    float ms = 0.0f;
                    check(c, cudaEventElapsedTime(&ms, e0, e1), "event time");
                    // the timing run leaves U modified: restore the spread state
                    for (int m = 0; m < L.M; ++m) copy_d2d(c, L.U + (long long)m * L.N, L.u0, L.N);
                    if (pick.first == 0 || ms < best) {
                        best = ms;
                        pick = cf;
                    }
                }
                configure(c, L, pick.first, pick.second);
                L.valid = false;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        check(c, cudaStreamSynchronize(c->stream), "sync");
        int flag = 0;
        check(c, cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "flag read");
        check(c, cudaMemset(c->d_err, 0, sizeof(int)), "memset");
        check(c, cudaMemset(c->d_stats, 0, ST_N * sizeof(long long)), "memset");
        check(c, cudaMemset(c->d_inst_iters, 0, c->inst.size() * sizeof(long long)), "memset");
        c->launches = 0;
        c->sweeps[0] = c->sweeps[1] = 0;
        if (flag & DEV_TIMEOUT) {
            cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned));
            return fail(c, SISDC_E_TIMEOUT, "a grid barrier wait timed out during tuning");
        }
    } catch (const Fail& f) {
        return f.st;
    }
    if (h_config) sisdc_ens_config(c, h_config);
    return SISDC_OK;
}

sisdc_status sisdc_ens_config(sisdc_ens c, int* h_config) {
    if (!c || !h_config) return SISDC_E_ARG;
    int k = 0;
    for (EnsGroup* g : c->groups)
        for (int which = 1; which >= 0; --which) {
            h_config[k++] = g->P;
            h_config[k++] = g->lv[which].P;
            h_config[k++] = g->lv[which].epb;
            h_config[k++] = g->lv[which].grid;
        }
    return SISDC_OK;
}

sisdc_status sisdc_ens_set_tiles(sisdc_ens c, int group, int fine, int epb, int grid) {
    if (!c || group < 0 || group >= (int)c->groups.size() || epb < 1 || grid < 1) return SISDC_E_ARG;
    EnsLevel& L = c->groups[group]->lv[fine ? 1 : 0];
    if (epb * L.Q > 512) return fail(c, SISDC_E_ARG, "a tile holds at most 512 nodes");
    try {
        check(c, cudaStreamSynchronize(c->stream), "sync");
        const int per = std::max(ens_occupancy(L.nq, L.mix ? 1 : 0, epb),
                                 ens_occupancy_capped(L.nq, L.mix ? 1 : 0, epb));
        if (per < 1 || grid > per * c->nsm) return fail(c, SISDC_E_ARG, "grid exceeds the co-resident blocks");
        configure(c, L, epb, grid);
        L.valid = false;
    } catch (const Fail& f) {
        return f.st;
    }
    return SISDC_OK;
}

int sisdc_ens_num_groups(sisdc_ens c) { return c ? (int)c->groups.size() : 0; }

const char* sisdc_ens_last_error(sisdc_ens c) { return c ? c->err.c_str() : "null ensemble"; }

}  // extern "C"
