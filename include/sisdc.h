/*
 * sisdc.h -- C ABI of the GB300 (sm_103a) semi-implicit multilevel SDC library.
 *
 * The library advances a system of conservation laws
 *     d_t u = f(u) = -div F_c(u) + (diffusion)                  (Sec. 2)
 * discretised by DG-SEM on periodic uniform meshes (Sec. 6) with the
 * semi-implicit multilevel spectral deferred correction method SI-MLSDC
 * (Sec. 3-4): incremental SI(1)/SI(2) sweeps over the collocation nodes
 * (Sec. 3.3, Algorithm 1), FAS coupling of space-time levels (Sec. 4.1,
 * eq. ml-cm:incremental:fas-mg:rhs), V-cycles (Algorithm 2) and Cascade/FMG
 * starts (Algorithms 3-4).  Every arithmetic step runs in CUDA kernels on
 * the GPU; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * State layout.  A solution on one level is a double array
 *     u[c][e][j][i]      c < ncomp, e = ey*nel_x + ex, j < NQY, i < NQ
 * with NQ = P+1 GLL nodes per direction (i fastest), NQY = NQ in 2D and 1
 * in 1D; N = nel * NQ * NQY nodes per component, NV = ncomp * N values.
 * An array over the collocation nodes m = 1..M of a level is U[m-1][NV]
 * (the node t_0 is not stored; u_0 is passed separately, Sec. 3.1).
 *
 * Memory.  Pointers named d_* are DEVICE pointers on the current CUDA
 * device, owned by the caller, and must stay valid until the work queued
 * on the context stream has finished.  Pointers named h_* are HOST
 * pointers, read or written synchronously.  Level work arrays are owned by
 * the library (allocated at sisdc_create_level, by cudaMalloc or by the
 * caller's allocator of sisdc_set_allocator, and released by sisdc_destroy).
 *
 * Streams and errors.  All device work is queued on the stream given to
 * sisdc_create and runs asynchronously; calls return after queuing.  Every
 * entry point returns a sisdc_status; on failure a message is available from
 * sisdc_last_error.  Conditions detected on the device (a CG solve that hit
 * its iteration cap, a non-finite residual, a grid-barrier timeout) are
 * recorded in a device flag and reported by the next sisdc_sync.  No C++
 * exception crosses the ABI.
 */
#ifndef SISDC_H
#define SISDC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sisdc_ctx_s* sisdc_ctx;
typedef struct sisdc_level_s* sisdc_level;
typedef struct sisdc_mlp_s* sisdc_mlp;

typedef enum {
    SISDC_OK = 0,
    SISDC_E_ARG = -1,       /* invalid argument                                  */
    SISDC_E_CUDA = -2,      /* CUDA runtime error                                */
    SISDC_E_NOCONV = -3,    /* an implicit solve reached cg_maxit                */
    SISDC_E_TIMEOUT = -4,   /* a bounded device wait gave up                     */
    SISDC_E_NONFINITE = -5, /* NaN/Inf met in a solve                            */
    SISDC_E_OOM = -6,       /* device allocation failed                          */
    SISDC_E_STATE = -7      /* call out of order (e.g. no level created)         */
} sisdc_status;

/* Collocation node sets (Sec. 3.1). */
typedef enum { SISDC_RADAU_RIGHT = 0, SISDC_LOBATTO = 1 } sisdc_nodes;

/* PDEs (Sec. 2 and the workloads): scalar convection-diffusion with constant
 * velocity adv, two-component viscous Burgers with flux u (x) u, 2D
 * compressible Euler with a perfect gas of ratio gamma, and 2D compressible
 * Navier-Stokes (Sec. 2.2: Newtonian stress with Stokes' hypothesis, Fourier
 * heat flux; units with gas constant 1, T = p / rho, viscosity mu,
 * conductivity mu gamma / ((gamma - 1) Pr)).  The Navier-Stokes viscous term
 * enters f explicitly, discretised by BR1 (lifted gradients of (v, T) with
 * central traces, central viscous face fluxes); the implicit term of the SI
 * integrators is nu_tilde L with nu_d = max(4/3, gamma / Pr) mu / rho_ref. */
typedef enum {
    SISDC_PDE_CONVDIFF = 0,
    SISDC_PDE_BURGERS = 1,
    SISDC_PDE_EULER = 2,
    SISDC_PDE_NS = 3
} sisdc_pde;

/* SISDC_FP64: every step in FP64.  SISDC_MIXED: operator applications and
 * CG matvecs in FP32; SDC residual, S.F quadrature, FAS tau, CG inner
 * products and the iterative-refinement residual of the implicit solve in
 * FP64.  Inputs and outputs are FP64 in both modes. */
typedef enum { SISDC_FP64 = 0, SISDC_MIXED = 1 } sisdc_precision;

/* Start strategies (Sec. 4.7): constant spread of u_0, predictor on all
 * levels, Cascade (Algorithm 3), FMG with one cycle per added level
 * (Algorithm 4; identical to Cascade for two levels). */
typedef enum {
    SISDC_START_SPREAD = 0,
    SISDC_START_PREDICTOR = 1,
    SISDC_START_CASCADE = 2,
    SISDC_START_FMG1 = 3
} sisdc_start;

/* One space-time level Q_l = Omega_l x T_l (Sec. 6.1): a periodic box
 * [lo, hi] split into nel[0] x nel[1] equal elements (nel[1] = 1 in 1D) of
 * degree P (1..8; 1..15 for 1D convection-diffusion in SISDC_FP64) and M
 * collocation nodes (1..8; >= 2 for Lobatto). */
typedef struct {
    int dim;
    int nel[2];
    int P;
    int M;
    int nodes;          /* sisdc_nodes */
    double lo[2];
    double hi[2];
} sisdc_level_desc;

typedef struct {
    int pde;            /* sisdc_pde                                          */
    int ncomp;          /* must match the PDE: 1, 2 or 4                      */
    double nu;          /* diffusivity nu (convdiff, Burgers)                 */
    double gamma;       /* ratio of specific heats (Euler)                    */
    double adv[2];      /* convection velocity (convdiff)                     */
    int precision;      /* sisdc_precision                                    */
    int si_stages;      /* 1 = SI(1), 2 = SI(2)  (Sec. 3.3)                   */
    double cg_rtol;     /* relative tolerance of the implicit solves          */
    int cg_maxit;       /* iteration cap of the implicit solves               */
    int Nc;             /* coarse sweeps per V-cycle (Algorithm 2; default 2) */
    int use_graph;      /* 1: sisdc_step replays a captured CUDA graph        */
    double mu;          /* dynamic viscosity 1/Re (Navier-Stokes)             */
    double Pr;          /* Prandtl number (Navier-Stokes)                     */
    double rho_ref;     /* reference density of nu_d (Navier-Stokes; > 0)     */
    int projection;     /* solution projection in space (Sec. 4.2): 0 embedded
                           interpolation, 1 L2 projection (I^T W I)^-1 I^T W
                           with the fine GLL quadrature                       */
    int fmg_cycles;     /* C_fmg: V-cycles per added level of the FMG start
                           (Algorithm 4); 0 means 1                           */
    int form;           /* 0: incremental (node-to-node) MLSDC; 1: the
                           non-incremental (zero-to-node) MLSDC of Sec. 4.5,
                           whose FAS right-hand side is built from F^0n
                           residuals (single-level sweeps are the same)       */
    int mixed_levels;   /* SISDC_MIXED only: bit l set = level l (creation
                           order, 0 = first created) uses the mixed form, the
                           others run in FP64; 0 = every level.  Levels whose
                           sweeps are barrier-latency bound (small coarse
                           levels) are often faster in FP64                    */
    double nu_tilde;    /* 0: nu_tilde = nu_d + dt_m/2 lam_max^2 per node and
                           sweep (Sec. 3.3, the diffusion-type coefficient of
                           the SI integrators); > 0: this constant instead
                           (the converged collocation result does not depend
                           on it; it changes the iteration only)            */
} sisdc_problem;

typedef struct {
    long long cg_solves;     /* implicit solves                               */
    long long cg_iters;      /* CG iterations summed over solves              */
    long long cg_max_iters;  /* largest iteration count of one solve          */
    long long cg_noconv;     /* solves that stopped at cg_maxit               */
    long long ir_steps;      /* iterative-refinement steps (SISDC_MIXED)      */
    long long sweeps[8];     /* correction/predictor sweeps per level index   */
    long long launches;      /* kernels launched by the library               */
} sisdc_stats;

/* --- context and levels --------------------------------------------------- */

/* Create a context bound to the current CUDA device and to the CUDA stream
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * problem struct is copied.  SISDC_E_ARG for an inconsistent problem. */
sisdc_status sisdc_create(const sisdc_problem* prob, void* cuda_stream, sisdc_ctx* out);
void sisdc_destroy(sisdc_ctx ctx);

/* Device allocator for the level work arrays (optional; the default is
 * cudaMalloc/cudaFree).  alloc(bytes, cuda_stream, user) returns device
 * memory of the context's device, at least 256-byte aligned and usable on
 * the context's stream, or NULL on failure (sisdc_create_level then returns
 * SISDC_E_OOM); release(ptr, bytes, cuda_stream, user) takes back exactly
 * what alloc returned, with the same size, at sisdc_destroy (after the
 * stream has finished).  This lets a caller's caching allocator (for
 * instance PyTorch's) own the memory.  Must be set before the first
 * sisdc_create_level (SISDC_E_STATE otherwise); both NULL restores the
 * default; exactly one NULL is SISDC_E_ARG.  The callbacks must outlive the
 * context. */
typedef void* (*sisdc_alloc_fn)(size_t bytes, void* cuda_stream, void* user);
typedef void (*sisdc_release_fn)(void* ptr, size_t bytes, void* cuda_stream, void* user);
sisdc_status sisdc_set_allocator(sisdc_ctx ctx, sisdc_alloc_fn alloc, sisdc_release_fn release, void* user);

/* Persson-Peraire artificial viscosity in f (Sec. 6, "Spatial
 * discretization": the diffusion matrix of the DG right-hand side
 * supplemented by an artificial viscosity; Sec. 8 uses it for the Burgers
 * moving front with d_s = c_s = 0.5 and for Sod's shock tube with d_s = 2,
 * c_s = 0.4).  The paper defers the form to its companion; this library's
 * reading: on every element the orthonormal-Legendre coefficients of the
 * sensor component `comp` (0 <= comp < ncomp; u_1 for Burgers, the density
 * for Euler) give s_e = log10(energy of the degree-P modes / total energy);
 * eps_e = c_s h/P lam_e r(s_e) with h the smaller element side, lam_e the
 * element's largest convective spectral radius and r = 0 below
 * s0 - d_s, 1 above s0 + d_s, (1 + sin(pi (s_e - s0) / (2 d_s))) / 2
 * between, s0 = log10(1/P^4).  f gains div(eps grad u) on every component
 * (BR1: derivatives lifted with central face values, scaled by eps_e, then
 * the divergence with central face values), evaluated at every state f is
 * evaluated at, and nu_tilde gains c_s h/P lam_max.  A correction sweep of
 * several iterations runs as single-sweep launches.  Must be called before
 * the first sisdc_create_level (SISDC_E_STATE otherwise); c_s = 0 switches
 * it off; d_s <= 0, c_s < 0 or a bad component is SISDC_E_ARG.  Levels then
 * hold M x nel + dim x M x ncomp x nodes more doubles.  Not available with
 * the learned sweep (sisdc_set_learned). */
sisdc_status sisdc_set_av(sisdc_ctx ctx, double d_s, double c_s, int comp);

/* Add a level (Sec. 6.1).  Levels must be added from coarse (l = 1) to fine
 * (l = L); adjacent levels must share the element grid (p-coarsening in
 * space, Sec. 6.2) and node kind (p-coarsening in time).  Work arrays are
 * allocated here (through the allocator of sisdc_set_allocator if one is
 * set; SISDC_E_OOM on failure).  The handle lives until sisdc_destroy. */
sisdc_status sisdc_create_level(sisdc_ctx ctx, const sisdc_level_desc* desc, sisdc_level* out);

/* Sizes of a level: components, nodes per component N, collocation nodes M. */
sisdc_status sisdc_level_info(sisdc_level lv, int* ncomp, long long* nodes, int* M);

/* Physical coordinates of the level's GLL nodes in the state layout
 * (h_x, h_y: host arrays of N doubles; h_y may be NULL in 1D). */
sisdc_status sisdc_level_coords(sisdc_level lv, double* h_x, double* h_y);

/* The library's own tables for this level (host arrays, each may be NULL):
 * collocation nodes tau[M] on [0,1]; node-to-node weights
 * w^nn[M*M] (Sec. 3.2, eq. nn_weights, row m = node); GLL nodes gll[NQ],
 * weights w[NQ] and differentiation matrix D[NQ*NQ] (row-major). */
sisdc_status sisdc_level_tables(sisdc_level lv, double* h_tau, double* h_wnn,
                                double* h_gll, double* h_w, double* h_D);

/* --- single operators (for verification and external drivers) ------------- */

/* d_c = c(d_u) = -div F_c(u): strong-form DG-SEM convective operator with a
 * Rusanov (local Lax-Friedrichs) face flux (Sec. 2, Sec. 6). */
sisdc_status sisdc_apply_conv(sisdc_level lv, const double* d_u, double* d_c);

/* d_Lu = L d_u with L = -M^{-1} A, A the SIPG stiffness (per component). */
sisdc_status sisdc_apply_lap(sisdc_level lv, const double* d_u, double* d_Lu);

/* d_out = f(d_u), the full right-hand side of the PDE on this level (Sec. 2):
 * c(u) plus nu L u (convection-diffusion, Burgers) or plus the BR1 viscous
 * term (Navier-Stokes).  Device arrays [ncomp][nel][Q].  Runs the persistent
 * sweep kernel on the level's work arrays, whose caches it invalidates (the
 * next sweep refreshes them). */
sisdc_status sisdc_apply_f(sisdc_level lv, const double* d_u, double* d_out);

/* Solve (I - c L) x = rhs, i.e. (M + c A) x = M rhs, by Jacobi-preconditioned
 * CG; d_x holds the initial guess on entry and the solution on exit.  The
 * iteration count is written to *h_iters (synchronises the stream) when
 * h_iters is not NULL. */
sisdc_status sisdc_solve(sisdc_level lv, double c, const double* d_rhs, double* d_x, int* h_iters);

/* The same solve with the element-wise fast-diagonalisation preconditioner
 * in place of Jacobi (the paper runs its implicit solves with PCG or a fast
 * diagonalisation solver, Sec. 8 "Runtime analysis"; the element-wise form
 * is this library's reading).  On the uniform periodic mesh the SIPG
 * stiffness is a Kronecker sum of 1D line operators; dropping the coupling
 * to neighbour elements leaves per element the block
 * B_e = M_y(x)M_x + c (M_y(x)K_x + K_y(x)M_x), inverted exactly through the
 * generalised eigenvectors of (K_x, M_x) and (K_y, M_y): four contractions
 * of length P+1 per node per CG iteration.  Stopping rule as sisdc_solve
 * with D^-1 replaced by B^-1.  Arguments, layout and errors as sisdc_solve;
 * uses the level's work arrays. */
sisdc_status sisdc_solve_fds(sisdc_level lv, double c, const double* d_rhs, double* d_x, int* h_iters);

/* No-allocation solve (the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory when they need a solve -- for
 * instance code that must stay inside a fixed memory budget owned by another
 * framework's caching allocator, or a time-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation).  It solves the same system
 * as sisdc_solve, (I - c L) x = rhs on the uniform periodic mesh described
 * by *desc (its M and nodes fields are ignored) with ncomp components, by
 * the same Jacobi-PCG kernel, but needs no context and no level: every
 * piece of scratch lives in one static device array of
 * SISDC_NOALLOC_SCRATCH_BYTES (16 MiB) that each GPU loading the library
 * holds until the process exits.  It calls no cudaMalloc/cudaFree; the
 * driver commits the array when it loads the library's code on a device,
 * which under CUDA's default lazy module loading happens at the first call
 * on that device (that call may then take memory and synchronise, the later
 * ones do not): make that first call at set-up time.
 *   - Fits when 5 * NV doubles (NV = ncomp * nodes) plus face traces and
 *     tables fit in the array (e.g. 2 x 32x32 elements of P = 7); larger
 *     problems are rejected with SISDC_E_ARG and a message in h_err.
 *   - d_x holds the initial guess on entry and the solution on exit
 *     (device pointers); the call is synchronous on cuda_stream and writes
 *     the CG iteration count to *h_iters (may be NULL).  h_err (may be
 *     NULL) receives a message of at most h_err_len bytes.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the
 *     caller.  Each call clears the parts that must start at zero. */
#define SISDC_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
sisdc_status sisdc_solve_noalloc(const sisdc_level_desc* desc, int ncomp, double c, const double* d_rhs,
                                 double* d_x, double rtol, int maxit, void* cuda_stream, int* h_iters,
                                 char* h_err, int h_err_len);

/* --- the method ------------------------------------------------------------ */

/* SI(1)/SI(2) predictor sweep (Sec. 3.3, eqs. sdc:incremental_predictor_si1
 * and _si2): fills d_U[M][NV] from d_u0[NV] over the slab of length dt. */
sisdc_status sisdc_predict(sisdc_level lv, const double* d_u0, double* d_U, double dt);

/* nsweeps incremental SI-MLSDC correction sweeps (Algorithm 1,
 * eq. ml-sdc:incremental) on d_U[M][NV] in place, with FAS right-hand side
 * d_g[M][NV] (NULL = 0).  Each call starts from f(d_U) of its input. */
sisdc_status sisdc_sweep(sisdc_level lv, const double* d_u0, double* d_U, const double* d_g,
                         double dt, int nsweeps);

/* FAS residual d_r = g - F^nn(U) (Sec. 4.3, eq. MLSDC:incremental:residual),
 * F^nn_m(U) = U_m - U_{m-1} - dt sum_i w^nn_{m,i} f(U_i), U_0 = u_0. */
sisdc_status sisdc_residual(sisdc_level lv, const double* d_u0, const double* d_U,
                            const double* d_g, double dt, double* d_r);

/* Space-time transfer between a level and the next finer one (Sec. 4.2,
 * Sec. 6.2).  op: 0 = interpolation I (coarse d_in[Mc] -> fine d_out[Mf]),
 * 1 = solution projection P (fine -> coarse, embedded interpolation),
 * 2 = residual restriction R = I^T (fine -> coarse), 3 = projection of one
 * state in space only (fine d_in[NV_f] -> coarse d_out[NV_c]). */
sisdc_status sisdc_transfer(sisdc_level fine, sisdc_level coarse, int op,
                            const double* d_in, double* d_out);

/* One MLSDC V-cycle (Algorithm 2) over all levels of the context with N_c
 * coarse sweeps.  The finest level's iterate d_U[M][NV] (and its initial
 * value d_u0) are caller-owned; coarse levels use library storage. */
sisdc_status sisdc_vcycle(sisdc_ctx ctx, const double* d_u0, double* d_U, double dt, int Nc);

/* One time step of length dt (Sec. 4.7): start strategy `start`
 * (sisdc_start), ncycles V-cycles, and a final fine post-sweep when
 * post_sweep != 0; d_u[NV] (finest level) holds u(t) on entry and
 * u(t+dt) = u_{L,M} on exit.  With a single level this is single-level SDC:
 * predictor plus ncycles sweeps.  t is the time at the start of the step
 * (unused by the autonomous PDEs supported here). */
sisdc_status sisdc_step(sisdc_ctx ctx, double* d_u, double t, double dt, int ncycles,
                        int start, int post_sweep);

/* Diagnostics of a state d_u[NV] (Sec. 7-8 report L2 errors per level): per
 * component c the GLL-quadrature L2 norm of u - ref (ref = d_ref, or 0 when
 * NULL), sqrt(sum_e sum_ij J w_i w_j (u - ref)^2), the discrete mass
 * sum_e sum_ij J w_i w_j u, and max |u - ref|.  Deterministic reduction
 * order; synchronous; host arrays of ncomp doubles (each may be NULL). */
sisdc_status sisdc_norms(sisdc_level lv, const double* d_u, const double* d_ref, double* h_l2,
                         double* h_mass, double* h_maxabs);

/* Wait for the context stream; report device-side conditions (NOCONV,
 * TIMEOUT, NONFINITE) recorded since the previous sisdc_sync and clear them. */
sisdc_status sisdc_sync(sisdc_ctx ctx);

/* Tile-shape autotuner of the persistent sweep kernel (not in the paper).
 * For every level, candidate shapes (elements per tile -> a block of
 * (P+1)^dim threads per element, and the number of persistent blocks) each run
 * one cache refresh and `reps` timed correction sweeps from the state d_u
 * (the fine-level state [ncomp][nel][Q]; projected to coarser levels and
 * spread over the collocation nodes; d_u is not modified); the fastest shape
 * is kept for all later launches.  h_config (nullable) receives 3 ints per
 * level, coarse to fine: elements per tile, blocks, threads per block.
 * Synchronous; invalidates a captured step graph; resets the counters. */
sisdc_status sisdc_autotune(sisdc_ctx ctx, const double* d_u, double dt, int reps, int* h_config);
/* The current shape of a level's sweep launches (any pointer may be NULL). */
sisdc_status sisdc_level_config(sisdc_level lv, int* h_epb, int* h_grid, int* h_block);

/* Counters since creation or the last reset (synchronises the stream). */
sisdc_status sisdc_get_stats(sisdc_ctx ctx, sisdc_stats* out);
sisdc_status sisdc_reset_stats(sisdc_ctx ctx);

/* Measurement hook.  When enabled (eager mode only: use_graph = 0), every
 * launch of the persistent correction-sweep kernel on level index `level`
 * (-1 = all levels) is bracketed by CUDA events on the context stream and
 * its CG iteration count is recorded.  sisdc_get_kernel_timing synchronises
 * the stream, returns the summed kernel time in ms, the number of timed
 * launches, their summed CG iterations, sum(iterations * NV of the level)
 * and the DOF-sweeps they performed (sum of nsweeps * NV), and restarts the
 * count. */
sisdc_status sisdc_set_kernel_timing(sisdc_ctx ctx, int enable, int level);
sisdc_status sisdc_get_kernel_timing(sisdc_ctx ctx, double* h_ms_total, long long* h_launches,
                                     long long* h_iters, long long* h_nodes_x_iters, long long* h_dof_sweeps);

/* --- learned initial guess / preconditioner of the implicit stage ----------
 * Not in the paper: an element-patch perceptron predicts, from the 3x3
 * element patch of a nodal residual field r (scaled by its RMS s, plus the
 * feature 0.1 log(c / h^2)), the correction of the centre element,
 * z = r_centre + s MLP(r_patch / s) (the residual itself is the exact
 * correction as c -> 0; the network learns the deviation);
 * per element and component, n_in = 9 Q + 1 -> hidden -> hidden (tanh) -> Q.
 * bf16 = 1: BF16 weights, and every GEMM multiplies BF16 operands on the
 * tensor cores with FP32 accumulation; bf16 = 0: FP32 weights and FP32 GEMMs
 * (the reference form).  FP32 master copy and Adam for training.  2D levels
 * with n_in <= 1024 (P <= 9); SISDC_E_ARG otherwise. */
sisdc_status sisdc_mlp_create(sisdc_level lv, int hidden, unsigned long long seed, int bf16, sisdc_mlp* out);
void sisdc_mlp_destroy(sisdc_mlp mlp);
sisdc_status sisdc_mlp_info(sisdc_mlp mlp, int* n_in, int* hidden, int* n_out, long long* nparam);
/* Parameters [W1 (n_in x H) | b1 | W2 (H x H) | b2 | W3 (H x Q) | b3], row-major FP32 master copy;
 * either pointer may be NULL (synchronous). */
sisdc_status sisdc_mlp_params(sisdc_mlp mlp, float* h_get, const float* h_set);
/* Loss 0.5 mean (MLP(x) - (dx - r)/s)^2 over all elements/components/nodes of one
 * logged solve (nodal residual d_r = b - (x0 - c L x0), correction d_dx,
 * coefficient c) and its gradient (host arrays; synchronous; no update). */
sisdc_status sisdc_mlp_loss_grad(sisdc_mlp mlp, const double* d_r, const double* d_dx, double c, double* h_loss,
                                 float* h_grad);
/* epochs of Adam steps, one step per logged solve k (d_r + k NV, d_dx + k NV,
 * h_c[k]); *h_loss = mean loss of the last epoch. */
sisdc_status sisdc_mlp_train(sisdc_mlp mlp, const double* d_r, const double* d_dx, const double* h_c, int nsolves,
                             int epochs, double lr, double* h_loss);
/* d_z (+)= r + s MLP(r / s) for every element and component (add != 0 adds). */
sisdc_status sisdc_mlp_apply(sisdc_mlp mlp, const double* d_r, double c, double* d_z, int add);
/* Forward-pass kernel of sisdc_mlp_apply in the BF16 mode: enable != 0 (the
 * default where it fits) = one fused persistent kernel on the tcgen05 tensor
 * cores -- the patch rows gathered straight into swizzled shared-memory
 * operand panels, the BF16 weights resident in shared memory (TMA), the FP32
 * accumulators in tensor memory, bias + tanh and the output z fused into
 * the epilogues; enable = 0: the patch matrix, three warp-level mma.sync
 * GEMMs and a scatter kernel.  SISDC_E_ARG when the fused kernel does not
 * fit the network (FP32 mode; hidden width not a multiple of 16 or above
 * 128; more than 128 outputs). */
sisdc_status sisdc_mlp_set_tc(sisdc_mlp mlp, int enable);
/* Synchronise the model's stream; SISDC_E_TIMEOUT if a bounded wait of the
 * fused forward pass gave up (its output is then invalid). */
sisdc_status sisdc_mlp_sync(sisdc_mlp mlp);
const char* sisdc_mlp_last_error(sisdc_mlp mlp);

/* Log, for every implicit solve of the FP64 form on level index `level`, the
 * initial nodal residual b - (x0 - c L x0) into d_r[k][NV], the correction x - x0
 * into d_dx[k][NV] and c into d_c[k] (k < capacity); NULL d_r disables.
 * Resets the count; sisdc_get_solve_log_count returns it (synchronous). */
sisdc_status sisdc_set_solve_log(sisdc_ctx ctx, int level, double* d_r, double* d_dx, double* d_c, int capacity);
sisdc_status sisdc_get_solve_log_count(sisdc_ctx ctx, int* h_count);

/* Learned initial guess inside the method (not in the paper): with mlp set
 * (a model created for this level), every correction sweep of level index
 * `level` (Algorithm 1, SI(1)/SI(2), FP64) runs composed from the
 * single-operation kernels instead of the persistent sweep kernel, and
 * before each implicit solve adds the network's correction of the nodal
 * residual of the warm start, x0 = u^{k-1}_m + z (sisdc_mlp_apply), then
 * runs Jacobi-PCG from x0 to the same cg_rtol: the result is the plain
 * method's to the solver tolerance, the CG iteration count is what changes
 * (sisdc_get_stats).  The network's scalar feature uses c = dt_m nu_tilde of
 * lambda(u0) (read once per sweep; the solve uses its exact c).  mlp = NULL
 * restores the persistent kernel.  SISDC_E_ARG for a mixed-precision level,
 * SISDC_E_STATE when the context captures CUDA graphs (the sweep reads
 * lambda on the host).  The caller keeps the model alive while it is set. */
sisdc_status sisdc_set_learned(sisdc_ctx ctx, int level, sisdc_mlp mlp);

/* Solve (I - c L) x = rhs to the context's cg_rtol: mode 0 = Jacobi-PCG from
 * d_x (as sisdc_solve); mode 1 = d_x += MLP(nodal residual), then PCG;
 * mode 2 = flexible CG (Polak-Ribiere) preconditioned by the MLP after the
 * same initial guess, with Jacobi-PCG warm-started from the current iterate
 * as the fallback on breakdown.  *h_iters = CG iterations (synchronous). */
sisdc_status sisdc_solve_learned(sisdc_level lv, sisdc_mlp mlp, double c, const double* d_rhs, double* d_x, int mode,
                                 int* h_iters);

/* --- batched ensemble of independent convection-diffusion problems ---------
 *
 * Many independent instances of u_t + a . grad u = nu lap u (Sec. 2, the
 * scalar convection-diffusion case) on the periodic unit square, each with
 * its own element grid, degree P, velocity a, viscosity nu and time step,
 * advanced together by two-level SI-MLSDC steps (Algorithm 2; Cascade start,
 * Algorithm 3, or the predictor start).  The coarse level of an instance has
 * degree ceil(P/2) on the same element grid (p-coarsening, Sec. 6.2) and Mc
 * collocation nodes of the same kind.  Instances of one degree share one
 * persistent cooperative launch per sweep; every instance keeps its own
 * implicit solves (own CG coefficients and stopping test), so the results
 * are those of solving the instances one by one. */
typedef struct sisdc_ens_s* sisdc_ens;

typedef struct {
    int nel[2];          /* elements in x and y (>= 1; nel[0] * nel[1] <= 2^24)  */
    int P;               /* fine polynomial degree, 2..8                         */
    double nu;           /* viscosity (>= 0)                                     */
    double adv[2];       /* velocity                                             */
    double dt;           /* time step (> 0)                                      */
} sisdc_ens_instance;

typedef struct {
    int M, Mc;           /* fine / coarse collocation nodes (1 <= Mc <= M <= 8)  */
    sisdc_nodes nodes;
    sisdc_precision precision;   /* SISDC_MIXED: FP32 inner CG for P >= 3 levels */
    int si_stages;       /* 1 or 2                                                */
    double cg_rtol;
    int cg_maxit;
    int Nc;              /* coarse sweeps per V-cycle                             */
    int ncycles;         /* V-cycles per step                                     */
    int start;           /* SISDC_START_CASCADE or SISDC_START_PREDICTOR          */
    int post_sweep;      /* final fine sweep after the last cycle                 */
    int use_graph;       /* capture one ensemble step as a CUDA graph             */
    int mixed_levels;    /* SISDC_MIXED only: bit 0 = coarse level, bit 1 = fine
                            level run the mixed form, the other FP64; 0 = both  */
} sisdc_ens_opts;

/* Create an ensemble of n instances on the current device and the stream
 * `cuda_stream` (NULL = legacy stream).  All work arrays are allocated here
 * (about 8 M + 4 doubles per fine node plus 8 Mc + 4 per coarse node).
 * SISDC_E_ARG for an invalid instance or option. */
sisdc_status sisdc_ens_create(const sisdc_ens_instance* inst, int n, const sisdc_ens_opts* opts, void* cuda_stream,
                              sisdc_ens* out);
void sisdc_ens_destroy(sisdc_ens ens);

/* Packed state layout: instance k occupies doubles offsets[k] ..
 * offsets[k] + nel[0] nel[1] (P+1)^2 - 1 of the state vector, as
 * [ey][ex][j][i] (GLL nodes, i fastest); *total = length of the vector.
 * Either pointer may be NULL. */
sisdc_status sisdc_ens_layout(sisdc_ens ens, long long* h_offsets, long long* h_total);

/* Node coordinates of the packed state (host arrays of *total doubles, as
 * sisdc_ens_layout): instance k's node (ey, ex, j, i) sits at
 * x = (ex + (xi_i + 1)/2) / nel[0], y = (ey + (xi_j + 1)/2) / nel[1] on the
 * unit square, xi the GLL nodes of its degree (Sec. 6).  For evaluating
 * initial data and exact solutions at the nodes.  h_y may be NULL. */
sisdc_status sisdc_ens_coords(sisdc_ens ens, double* h_x, double* h_y);

/* Advance every instance by nsteps steps of its own dt; d_u = packed state
 * (device, caller-owned), updated in place.  Asynchronous on the stream. */
sisdc_status sisdc_ens_step(sisdc_ens ens, double* d_u, int nsteps);

/* Tile-shape autotuner: for every level of every degree group, times
 * `nsweeps` correction sweeps from the state d_u (spread over the nodes) for
 * each candidate (elements per tile, blocks per SM, including the
 * register-capped build's larger block counts) and keeps the fastest.
 * d_u is not modified.  h_config (nullable) receives the result as for
 * sisdc_ens_config.  Synchronous. */
sisdc_status sisdc_ens_autotune(sisdc_ens ens, const double* d_u, int nsweeps, int* h_config);
/* Current tile shapes: per group and level (fine, then coarse) the 4 ints
 * (group degree, level degree, elements per tile, blocks in the grid);
 * h_config holds 8 * sisdc_ens_num_groups(ens) ints. */
sisdc_status sisdc_ens_config(sisdc_ens ens, int* h_config);
int sisdc_ens_num_groups(sisdc_ens ens);
/* Set the tile shape of one level (fine != 0: fine level) of group `group`
 * (groups in increasing degree): epb elements per tile (epb (P+1)^2 <= 512
 * threads), `grid` persistent blocks (at most the co-resident count; fewer
 * when the level has fewer tiles).  Each kernel is built twice: for up to 128
 * registers per thread and capped at 64; a grid with more blocks than the
 * first build keeps resident on the SMs runs the capped build (the
 * co-resident count above is the larger of the two).  The order of the
 * per-instance partial sums follows the grid, so results of different grids
 * agree to rounding.  Synchronous. */
sisdc_status sisdc_ens_set_tiles(sisdc_ens ens, int group, int fine, int epb, int grid);

/* Synchronise and report device error flags (as sisdc_sync). */
sisdc_status sisdc_ens_sync(sisdc_ens ens);
/* Counters (synchronous): sweeps[0] / sweeps[1] = coarse / fine sweeps
 * (counted per group launch); h_inst_iters (nullable, n entries) = fine-level
 * CG iterations of each instance. */
sisdc_status sisdc_ens_get_stats(sisdc_ens ens, sisdc_stats* out, long long* h_inst_iters);
sisdc_status sisdc_ens_reset_stats(sisdc_ens ens);

/* Measurement hook: with enable != 0, every fine-level correction-sweep
 * launch of every group is bracketed by CUDA events on the ensemble's
 * stream (eager mode only: SISDC_E_STATE when use_graph is set).
 * sisdc_ens_get_kernel_timing (synchronous) returns, per group (in
 * increasing degree; arrays of sisdc_ens_num_groups entries, nullable), the
 * summed launch time in ms and the number of launches since the hook was
 * enabled or last read, and clears them. */
sisdc_status sisdc_ens_set_kernel_timing(sisdc_ens ens, int enable);
sisdc_status sisdc_ens_get_kernel_timing(sisdc_ens ens, double* h_ms, long long* h_launches);
const char* sisdc_ens_last_error(sisdc_ens ens);

/* --- stability function on the Dahlquist problem (Sec. 5) -----------------
 *
 * R(z) of one SI-MLSDC step for u' = z u with the semi-implicit split of the
 * Fourier-mode problem (Sec. 5): Im(z) convective (explicit), Re(z) diffusive
 * (implicit, nu_d = -Re(z)), nu_tilde = -Re(z) + dt_m/2 Im(z)^2, dt = 1,
 * u(0) = 1.  Levels coarsen in time only (node counts M[0] <= ... , coarse
 * to fine).  One GPU thread per point. */
typedef struct {
    int nlevels;         /* 1..4                                               */
    int M[4];            /* collocation nodes per level, coarse to fine        */
    sisdc_nodes nodes;
    int si_stages;       /* 1 or 2                                             */
    int ncycles;         /* V-cycles (one level: correction sweeps)            */
    int start;           /* sisdc_start                                        */
    int post_sweep;
    int Nc;              /* coarse sweeps per V-cycle                          */
    int fmg_cycles;      /* C_fmg of the FMG start (0 means 1)                 */
} sisdc_stab_opts;
/* d_z: [n][2] (Re, Im) device array; d_R: [n][2] receives R(z).
 * Asynchronous on `cuda_stream` (a cudaStream_t; NULL = legacy stream). */
sisdc_status sisdc_stability(const sisdc_stab_opts* opts, const double* d_z, double* d_R, long long n,
                             void* cuda_stream);

/* --- number-format conversions of the mixed-precision kernels ------------
 *
 * The mixed form's FP32 <-> FP64 and FP64 -> double-single conversions are
 * built from the IEEE-754 bit patterns with integer instructions (on GB300
 * the hardware conversions issue on the FP64 unit).  This entry applies them
 * elementwise so that they can be checked against the hardware conversions:
 *   kind 0: d_in double[n] -> d_out float[n], rounded to nearest (ties even)
 *   kind 1: d_in float[n]  -> d_out double[n], exact
 *   kind 2: d_in double[n] -> d_out float[2n], (hi, lo) double-single pairs:
 *           hi = the input truncated to 24 significand bits, lo = the
 *           remainder truncated to 24 bits (2^-74 <= |x| < 2^128; other
 *           inputs: hi = the rounded float, lo = the rounded remainder)
 *   kind 3: d_in float[2n] (hi, lo) -> d_out double[n] = hi + lo rounded
 * Device pointers, n >= 0, asynchronous on `cuda_stream`; SISDC_E_ARG for an
 * unknown kind, n < 0 or a null pointer with n > 0. */
sisdc_status sisdc_convert(int kind, const void* d_in, long long n, void* d_out, void* cuda_stream);

/* --- failure detection of the bounded grid barrier -------------------------
 *
 * Every persistent kernel synchronises its blocks with a grid barrier whose
 * wait is bounded (2 s of the global timer, or 2^24 polls); a block whose
 * wait runs out records SISDC_E_TIMEOUT for sisdc_sync and leaves the
 * kernel, so the context stays usable.  This entry exercises that path:
 * it launches a cooperative kernel of `nblocks` blocks (1..number of SMs)
 * that meet at one barrier, except block `absent` (absent < 0: none), which
 * never arrives; the other blocks' wait then runs out after `timeout_ms`
 * (1..2000).  Synchronous on `cuda_stream`.  Returns SISDC_OK if the
 * barrier completed, SISDC_E_TIMEOUT if the wait gave up, SISDC_E_ARG for
 * arguments out of range, SISDC_E_CUDA for launch errors. */
sisdc_status sisdc_barrier_selftest(int nblocks, int absent, double timeout_ms, void* cuda_stream);

/* Message of the last failing call on this context ("" if none). */
const char* sisdc_last_error(sisdc_ctx ctx);

#ifdef __cplusplus
}
#endif

#endif /* SISDC_H */
