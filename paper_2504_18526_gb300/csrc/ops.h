// Internal launch interface of the SI-MLSDC kernels (host side).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace sisdc {

// ---- SIPG diffusion (ops_sipg.cu) -------------------------------------------
enum ApplyMode : int { APPLY_A = 0, APPLY_LAP = 1, APPLY_LAP_F = 2, APPLY_OP = 3, APPLY_RES = 4, APPLY_RESN = 5 };

struct ApplyArgs {
    Geo g;
    const double* u;
    const double* tr;     // traces of u (from launch_traces)
    double* out;
    double* out2;         // APPLY_LAP_F: F = cc + nu * Lu
    const double* cc;     // APPLY_LAP_F: c cache; APPLY_RES: right-hand side
    double nu;
    Coef c;               // APPLY_OP: Mass u + c A u; APPLY_RES: Mass rhs - (Mass u + c A u)
    int mode;
};

struct PCGArgs {
    Geo g;
    double* x;            // initial guess in, solution out
    double* r;
    double* p;
    double* Ap;
    double* trx;          // trace buffer for x
    double* trp;          // trace buffer for p
    int nterms;           // right-hand side b = sum_t coef_t * in_t (nodal)
    const double* in[MAXTERMS];
    Coef coef[MAXTERMS];
    Coef cimp;            // system (M + c A) x = M b
    double* part;         // 4 * gridDim partial sums
    unsigned* bar_count;
    unsigned* bar_exit;
    int* err;
    long long* stats;
    double rtol;
    int maxit;
    int* iters_out;       // iteration count of this solve (nullable)
    int prec;             // PCG_JACOBI, or PCG_FDS (element-wise fast diagonalisation, g.fds)
    double* z;            // PCG_FDS: preconditioned residual B^-1 r
};
enum PcgPrec : int { PCG_JACOBI = 0, PCG_FDS = 1 };

cudaError_t launch_traces(const Geo& g, const double* u, double* tr, cudaStream_t s);
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s);
// out = M^-1 in per node (GLL mass), all components
cudaError_t launch_minv(const Geo& g, const double* in, double* out, cudaStream_t s);
// Grid size for the cooperative PCG kernel of this geometry (0 if unsupported).
int pcg_grid(const Geo& g, int* block);
cudaError_t launch_pcg(const PCGArgs& a, int grid, int block, cudaStream_t s);

// ---- convective operator (ops_conv.cu) -------------------------------------
enum ConvMode : int { CONV_OUT = 0, CONV_DELTA = 1 };

struct ConvArgs {
    Geo g;
    int pde;              // sisdc_pde
    double gamma;
    double ax, ay;
    const double* u;
    double* out;          // c(u) (CONV_OUT, or also in CONV_DELTA when not null)
    double* cache;        // CONV_DELTA: delta = c - cache; cache = c
    double* delta;
    double* lam;          // max spectral radius (atomic max), may be null
    int mode;
};
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s);

// ---- persistent sweep kernel (sweep.cuh, sweep_*.cu) ------------------------
// SW_FEVAL: f(u0) into fout (one state; uses the level's work arrays)
enum SweepMode : int { SW_REFRESH = 0, SW_PREDICT = 1, SW_CORRECT = 2, SW_FEVAL = 3 };

struct SweepArgs {
    Geo g;
    int pde;
    double gamma, ax, ay;   // flux parameters
    double nu;              // physical diffusion in f
    double nu_d;            // nu_d of nu_tilde = nu_d + dt_m/2 lam_max^2
    double nu_tilde_fix;    // > 0: constant nu_tilde instead of the formula
    double nu_lam;          // artificial viscosity's share of nu_tilde per unit of lam_max (c_s h / P)
    double mu, kappa;       // Navier-Stokes viscosity and heat conductivity
    double* FV;             // Navier-Stokes viscous flux scratch [6][N]: F_v^x, F_v^y of
                            // the momentum and energy components
    double* fout;           // SW_FEVAL output [NV]
    int mode, nsweeps, stages, M;
    double dt;
    double dtau[MMAX];
    double W[MMAX * MMAX];  // w^nn, row m
    const double* u0;
    double* U;              // [M][NV]
    const double* G;        // FAS right-hand side [M][NV] or null
    int mix;                // 1: mixed precision (caches and inner CG in FP32)
    double* F;              // cached f [M][NV] (FP64)
    void *CC, *LU;          // cached c and L u [M][NV] (FP64, or FP32 when mix)
    double* Qb;             // S.F quadrature [M][NV] (FP64)
    void *c0, *dC, *tmpc;   // [NV] (FP64, or FP32 when mix)
    double* r;              // CG residual, or M b of the refinement (FP64) [NV]
    void *p, *p2, *Ap;      // CG vectors (FP64, or FP32 when mix) [NV]
    void* rf;               // inner FP32 residual of the refinement (mix); FP64 form: z = D^-1 r [NV]
    double* lam;            // [2][MMAX+1] spectral radius slots (old, new)
    double* part;           // 8 * grid partial sums
    double* partmax;        // (MMAX+1) * grid partial maxima
    unsigned* bar_count;
    unsigned* bar_exit;
    int* err;
    long long* stats;
    double rtol;
    int maxit;
    int epb;
    int* iters_out;         // CG iterations of this launch (summed over its solves; nullable)
    // solve log (FP64 form): for every implicit solve, the initial nodal
    // residual b - (x0 - c L x0) and the correction x - x0 into slot k of log_r /
    // log_dx ([cap][NV]) and c into log_c[k]; k counts on from *log_count.
    double* log_r;
    double* log_dx;
    double* log_c;
    int* log_count;
    int log_cap;
    cudaStream_t stream;
};
// returns the largest cooperative grid (0 if unavailable) for tiles of *epb
// elements per block (in: requested size, 0 = default heuristic; out: used)
int sweep_config(const Geo& g, int pde, int mix, int* epb, int* block);
cudaError_t launch_sweep(const SweepArgs& a, int grid, int block);

// ---- elementwise and transfer kernels (ops_misc.cu) -------------------------
struct LinArgs {          // out[idx] = sum_t coef_t * in_t[idx], idx < n
    long long n;
    int nterms;
    const double* in[MAXTERMS];
    Coef coef[MAXTERMS];
    double* out;
};
cudaError_t launch_lincomb(const LinArgs& a, cudaStream_t s);

// Q[m] = dt * sum_i W[m][i] F[i] for m < M (arrays of n values; F in FP32
// when f32, accumulation in FP64 either way)
cudaError_t launch_quad(const void* F, int f32, double* Q, const double* W, int M, double dt,
                        long long n, cudaStream_t s);

// r[m] = (g ? g[m] : 0) - (U[m] - U[m-1] - Q[m]),  U[-1] = u0   (sign = +1)
// r[m] = U[m] - U[m-1] - Q[m]                                     (sign = 0, g ignored)
cudaError_t launch_fnn(const double* u0, const double* U, const double* Q, const double* g,
                       double* r, int M, long long n, int residual, cudaStream_t s);

struct TransferArgs {
    int dim, nqi, nqo, Mi, Mo, ncomp, nel;
    const double* S;      // [nqo*nqi] per-direction space matrix (device)
    const double* Tt;     // [Mo*Mi] time matrix (device)
    const double* in;     // [Mi][ncomp][nel][nqi^dim]
    double* out;          // [Mo][ncomp][nel][nqo^dim]
    int add;              // out += instead of out =
    // 2:1 h-coarsening (rx or ry = 2; 0 or 1 = the same elements on both
    // sides, the fields below unused): per direction the child matrices
    // S [rx][nqo*nqi] (x) and Sy [ry][nqo*nqi] (y); c2f = coarse-to-fine
    // (each fine element takes its child's matrix applied to its coarse
    // element), else fine-to-coarse (each coarse element sums its children)
    int rx, ry, c2f;
    int nexi, neyi, nexo, neyo;
    const double* Sy;
};
cudaError_t launch_transfer(const TransferArgs& a, cudaStream_t s);

// ---- artificial viscosity (ops_av.cu) ----------------------------------------
// F_s += div(eps grad U_s) for the n states U_s (each [ncomp][N]), eps per
// element from the modal decay of component `comp` (Persson-Peraire)
struct AvArgs {
    Geo g;
    int pde;                // convective flux of the spectral radius (NS: Euler's)
    double gamma, ax, ay;
    int comp;               // sensor component
    double s0, kappa;       // sensor threshold log10(1/P^4) and ramp half-width d_s
    double eps_scale;       // c_s h / P
    const double* vinv;     // [nq*nq] nodal -> orthonormal Legendre coefficients
    const double* U;        // [n][ncomp*N]
    double* F;              // [n][ncomp*N], added to
    double* eps;            // [n][nel] scratch (the viscosities, kept for inspection)
    double* grad;           // [n][dim][ncomp*N] scratch
    int n;
};
cudaError_t launch_av(const AvArgs& a, cudaStream_t s);

// diagnostics: scratch holds partials and, at offset ncomp*NORM_BLOCKS*3,
// the result [ncomp][3] = (L2 norm of u - ref, mass of u, max |u - ref|)
int norms_scratch_doubles(int ncomp);
// deterministic dot products: out[0] = sum a b w, w = 1 or the Jacobi factor
// 1 / (mass + c diagA) of each node (jacobi != 0); scratch as for norms
cudaError_t launch_dot(const Geo& g, const double* a, const double* b, int jacobi, double c, double* scratch,
                       cudaStream_t s);
cudaError_t launch_norms(const Geo& g, const double* u, const double* ref, double* scratch, cudaStream_t s);

// ---- ensemble of independent 2D convection-diffusion problems (ens.cuh) ------
// One instance of an ensemble level: its elements are e0 .. e0 + nex*ney - 1
// of the level (row-major [ey][ex]), its tiles t0 .. t0 + nt - 1.  Copied
// into shared memory as 64-bit words: keep every member 8-byte sized or paired.
struct EnsInst {
    long long e0;
    int nex, ney;
    int t0, nt;
    double hx, hy, sx, sy, ihx, ihy, taux, tauy;
    double liftLx, liftRx, liftLy, liftRy;   // (2/h)/w_0, (2/h)/w_P
    double ax, ay, nu;
    double lam;                              // max(|a_x|, |a_y|)
    double dt;                               // the instance's time step
    double rho, irho;                        // h_y / h_x, h_x / h_y
    double mq, imq;                          // h_x h_y / 4 and its inverse (mass = mq w_i w_j)
};

// instance records a block keeps in shared memory for the whole launch
constexpr int ENS_LSMEM = 128;

struct EnsArgs {
    const EnsInst* inst;    // [ninst]
    int ninst;
    const int4* tiles;      // [ntiles] (instance, owner-local index, first element, elements)
    long long ntiles;
    int epb;                // elements per tile; the block has epb * Q threads
    const int* nloc;        // [grid] instances touched by each block
    const int* loc_inst;    // [grid][lmax] their indices
    int lmax;
    void* loc;              // [grid][lmax] per-block solve state
    double* loc_dinv;       // [grid][lmax][Q] per-block Jacobi factors
    float* loc_dinv32;      // [grid][lmax][Q] the same factors rounded to FP32 (mixed form)
    // FP64 CG face traces [element][face][value | derivative][NQ]: of z (tz) and of the
    // search direction (tp0 / tp1, alternating like p / p2); nullable: faces recomputed
    double *tz, *tp0, *tp1;
    long long N;            // nodes of the level
    const double *D, *K, *w, *dl;   // degree-P tables; dl = h * (diagonal of the 1D SIPG line operator)
    int mode, nsweeps, stages, M;
    double dtau[MMAX];
    double W[MMAX * MMAX];
    const double* u0;
    double* U;
    const double* G;
    double *F, *CC, *LU, *Qb, *c0, *dC, *tmpc;
    double* r;
    void *p, *p2, *Ap, *rf;
    double* part;           // (2 * 4 * ninst + 2) * grid partial sums
    unsigned* bar_count;
    unsigned* bar_exit;
    int* err;
    long long* stats;
    double rtol;
    int maxit;
    long long* inst_iters;  // [ninst] CG iterations per instance (nullable)
};
// blocks per SM of the ensemble kernel for tiles of epb elements (0: unavailable)
int ens_occupancy(int nq, int mix, int epb);
// the same for the kernel compiled for at most 64 registers per thread
int ens_occupancy_capped(int nq, int mix, int epb);
cudaError_t launch_ens_sweep(const EnsArgs& a, int nq, int mix, int grid, cudaStream_t s, int capped);

}  // namespace sisdc
