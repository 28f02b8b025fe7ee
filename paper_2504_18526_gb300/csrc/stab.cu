// Batched stability function of SI-MLSDC on the Dahlquist problem (Sec. 5).
//
// For a Fourier mode u = u_hat(t) e^{ikx} of u_t = -v u_x + nu u_xx (k = 1)
// the operators of the method reduce to scalars: c(u) = i Im(lam) u,
// L u = -u, f(u) = lam u, nu_d = -Re(lam), lam_max = |Im(lam)|, and the
// implicit solve (I - c L) x = r is x = r / (1 + c).  One thread runs one
// complete time step (dt = 1, u(0) = 1) for its z = lam: start strategy,
// V-cycles over the levels (time coarsening only), post-sweep; R(z) = u(1).
// The steps are those of the field solver (Algorithm 1 with the SI(1)/SI(2)
// deltas, Algorithm 2 with the FAS right-hand side, Algorithms 3 and 4).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/sisdc.h"
#include "common.cuh"
#include "tables.h"

namespace sisdc {

constexpr int STAB_LMAX = 4;

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }

// Per-level time tables: M, substeps dtau[m], w^nn row-major; transfers to
// the next coarser level (It: Mf x Mc, Pt: Mc x Mf, Rt = It^T: Mc x Mf).
struct StabLevel {
    int M;
    double dtau[MMAX];
    double W[MMAX * MMAX];
    double It[MMAX * MMAX], Pt[MMAX * MMAX], Rt[MMAX * MMAX];
};

struct StabArgs {
    const StabLevel* lv;   // [nlevels], coarse to fine
    int nlevels, stages, ncycles, start, post, Nc, fmg_cycles;
    const double* z;       // [n][2]
    double* R;             // [n][2]
    long long n;
};

struct Dahlquist {
    double lr, li;         // lam
    __device__ cplx conv(cplx u) const { return {-li * u.im, li * u.re}; }      // i Im(lam) u
    __device__ cplx f(cplx u) const { return conv(u) + lr * u; }                // lam u
    __device__ double nut(double dtm) const { return -lr + 0.5 * dtm * li * li; }
    __device__ cplx solve(double c, cplx r) const {     // (I - c L) x = r with L = -1
        const double d = 1.0 + c;
        return {r.re / d, r.im / d};
    }
};

struct StabStep {
    const StabArgs& a;
    Dahlquist p;
    cplx U[STAB_LMAX][MMAX], G[STAB_LMAX][MMAX], Vv[STAB_LMAX][MMAX];
    bool hasG[STAB_LMAX];

    __device__ StabStep(const StabArgs& args, double lr, double li) : a(args) { p = Dahlquist{lr, li}; }

    __device__ void predictor(int l) {
        const StabLevel& L = a.lv[l];
        cplx uprev{1.0, 0.0};
        for (int m = 0; m < L.M; ++m) {
            const double dtm = L.dtau[m];
            if (dtm == 0.0) {
                U[l][m] = uprev;
                continue;
            }
            const double c = dtm * p.nut(dtm);
            cplx x = p.solve(c, uprev + dtm * p.conv(uprev));
            if (a.stages == 2) x = p.solve(c, uprev + dtm * p.conv(x));
            U[l][m] = x;
            uprev = x;
        }
    }

    __device__ void corrector(int l, bool withG, int nsweeps) {
        const StabLevel& L = a.lv[l];
        const int M = L.M;
        for (int k = 0; k < nsweeps; ++k) {
            cplx Uold[MMAX], Q[MMAX];
            for (int m = 0; m < M; ++m) Uold[m] = U[l][m];
            for (int m = 0; m < M; ++m) {
                cplx s{0.0, 0.0};
                for (int i = 0; i < M; ++i) s = s + L.W[m * M + i] * p.f(Uold[i]);
                Q[m] = s;                                  // dt = 1
            }
            cplx unew_prev{1.0, 0.0};
            for (int m = 0; m < M; ++m) {
                const double dtm = L.dtau[m];
                const cplx uold_prev = m == 0 ? cplx{1.0, 0.0} : Uold[m - 1];
                cplx base = unew_prev + Q[m];
                if (withG) base = base + G[l][m];
                if (dtm == 0.0) {
                    U[l][m] = base;
                    unew_prev = base;
                    continue;
                }
                const double nu_new = p.nut(dtm), nu_old = p.nut(dtm);
                const cplx LUold = -1.0 * Uold[m];
                const cplx old1 = dtm * (p.conv(uold_prev) + nu_old * LUold);
                cplx x = p.solve(dtm * nu_new, base + dtm * p.conv(unew_prev) - old1);
                if (a.stages == 2) {
                    const cplx old2 = dtm * (p.conv(Uold[m]) + nu_old * LUold);
                    x = p.solve(dtm * nu_new, base + dtm * p.conv(x) - old2);
                }
                U[l][m] = x;
                unew_prev = x;
            }
        }
    }

    // F^nn_m(X) = X_m - X_{m-1} - sum_i w^nn_{m,i} f(X_i), X_0 = u0 = 1
    __device__ void fnn(int l, const cplx* X, cplx* out) const {
        const StabLevel& L = a.lv[l];
        for (int m = 0; m < L.M; ++m) {
            cplx s{0.0, 0.0};
            for (int i = 0; i < L.M; ++i) s = s + L.W[m * L.M + i] * p.f(X[i]);
            const cplx prev = m == 0 ? cplx{1.0, 0.0} : X[m - 1];
            out[m] = X[m] - prev - s;
        }
    }

    __device__ void interp_add(int l, const cplx* Xc, bool add) {     // U[l] (+)= It Xc
        const StabLevel& F = a.lv[l];
        const int Mc = a.lv[l - 1].M;
        for (int m = 0; m < F.M; ++m) {
            cplx s{0.0, 0.0};
            for (int n = 0; n < Mc; ++n) s = s + F.It[m * Mc + n] * Xc[n];
            U[l][m] = add ? U[l][m] + s : s;
        }
    }

    // Algorithm 2 on levels 0..top-1
    __device__ void vcycle(int top) {
        for (int l = 0; l < top; ++l) hasG[l] = false;
        for (int l = top - 1; l >= 1; --l) {
            corrector(l, hasG[l], 1);
            cplx r[MMAX];
            fnn(l, U[l], r);
            for (int m = 0; m < a.lv[l].M; ++m) r[m] = (hasG[l] ? G[l][m] : cplx{0.0, 0.0}) - r[m];
            const StabLevel& F = a.lv[l];
            const int Mc = a.lv[l - 1].M, Mf = F.M;
            for (int q = 0; q < Mc; ++q) {
                cplx s{0.0, 0.0};
                for (int m = 0; m < Mf; ++m) s = s + F.Pt[q * Mf + m] * U[l][m];
                Vv[l - 1][q] = s;
            }
            cplx fv[MMAX];
            fnn(l - 1, Vv[l - 1], fv);
            for (int q = 0; q < Mc; ++q) {
                cplx s{0.0, 0.0};
                for (int m = 0; m < Mf; ++m) s = s + F.Rt[q * Mf + m] * r[m];
                G[l - 1][q] = fv[q] + s;
                U[l - 1][q] = Vv[l - 1][q];
            }
            hasG[l - 1] = true;
        }
        corrector(0, hasG[0], a.Nc);
        for (int l = 1; l < top; ++l) {
            cplx d[MMAX];
            for (int q = 0; q < a.lv[l - 1].M; ++q) d[q] = U[l - 1][q] - Vv[l - 1][q];
            interp_add(l, d, true);
            if (l < top - 1) corrector(l, hasG[l], 1);
        }
    }

    __device__ cplx step() {
        const int L = a.nlevels;
        if (L == 1) {
            predictor(0);
            corrector(0, false, a.ncycles);
            return U[0][a.lv[0].M - 1];
        }
        if (a.start == SISDC_START_CASCADE || a.start == SISDC_START_FMG1) {
            predictor(0);
            corrector(0, false, 1);
            interp_add(1, U[0], false);
            for (int l = 1; l < L - 1; ++l) {
                if (a.start == SISDC_START_FMG1)
                    for (int c = 0; c < (a.fmg_cycles > 0 ? a.fmg_cycles : 1); ++c) vcycle(l + 1);
                else
                    corrector(l, false, 1);
                interp_add(l + 1, U[l], false);
            }
        } else if (a.start == SISDC_START_PREDICTOR) {
            for (int l = 0; l < L; ++l) predictor(l);
        } else {
            for (int l = 0; l < L; ++l)
                for (int m = 0; m < a.lv[l].M; ++m) U[l][m] = cplx{1.0, 0.0};
        }
        for (int k = 0; k < a.ncycles; ++k) vcycle(L);
        if (a.post) corrector(L - 1, false, 1);
        return U[L - 1][a.lv[L - 1].M - 1];
    }
};

__global__ void k_stability(const __grid_constant__ StabArgs a) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += (long long)gridDim.x * blockDim.x) {
        StabStep s(a, a.z[2 * t], a.z[2 * t + 1]);
        const cplx r = s.step();
        a.R[2 * t] = r.re;
        a.R[2 * t + 1] = r.im;
    }
}

}  // namespace sisdc

using namespace sisdc;

extern "C" sisdc_status sisdc_stability(const sisdc_stab_opts* o, const double* d_z, double* d_R, long long n,
                                        void* cuda_stream) {
    if (!o || !d_z || !d_R || n < 0) return SISDC_E_ARG;
    if (o->nlevels < 1 || o->nlevels > STAB_LMAX) return SISDC_E_ARG;
    if (o->nodes != SISDC_RADAU_RIGHT && o->nodes != SISDC_LOBATTO) return SISDC_E_ARG;
    if (o->si_stages != 1 && o->si_stages != 2) return SISDC_E_ARG;
    if (o->ncycles < 0 || o->Nc < 0 || o->start < 0 || o->start > 3 || o->fmg_cycles < 0) return SISDC_E_ARG;
    std::vector<StabLevel> hl(o->nlevels);
    std::vector<LevelTables> tab(o->nlevels);
    for (int l = 0; l < o->nlevels; ++l) {
        const int M = o->M[l];
        if (M < 1 || M > MMAX || (l > 0 && M < o->M[l - 1])) return SISDC_E_ARG;
        if (!build_level_tables(1, M, o->nodes == SISDC_LOBATTO, &tab[l])) return SISDC_E_ARG;
        StabLevel& s = hl[l];
        s = StabLevel{};
        s.M = M;
        for (int m = 0; m < M; ++m) s.dtau[m] = tab[l].dtau[m];
        for (int k = 0; k < M * M; ++k) s.W[k] = tab[l].wnn[k];
        if (l > 0) {
            const int Mc = o->M[l - 1];
            const std::vector<double> It = lagrange_matrix(tab[l - 1].tau, tab[l].tau);   // Mf x Mc
            const std::vector<double> Pt = lagrange_matrix(tab[l].tau, tab[l - 1].tau);   // Mc x Mf
            for (int k = 0; k < M * Mc; ++k) s.It[k] = It[k];
            for (int k = 0; k < Mc * M; ++k) s.Pt[k] = Pt[k];
            for (int q = 0; q < Mc; ++q)
                for (int m = 0; m < M; ++m) s.Rt[q * M + m] = It[m * Mc + q];
        }
    }
    if (n == 0) return SISDC_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    StabLevel* d_lv = nullptr;
    cudaError_t e = cudaMallocAsync(&d_lv, hl.size() * sizeof(StabLevel), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lv, hl.data(), hl.size() * sizeof(StabLevel), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        StabArgs a{};
        a.lv = d_lv;
        a.nlevels = o->nlevels;
        a.stages = o->si_stages;
        a.ncycles = o->ncycles;
        a.start = o->start;
        a.post = o->post_sweep ? 1 : 0;
        a.Nc = o->Nc;
        a.fmg_cycles = o->fmg_cycles;
        a.z = d_z;
        a.R = d_R;
        a.n = n;
        long long nb = (n + 127) / 128;
        if (nb > 152LL * 64) nb = 152LL * 64;
        k_stability<<<(unsigned)nb, 128, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (d_lv) {
        const cudaError_t f = cudaFreeAsync(d_lv, st);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SISDC_E_OOM : SISDC_E_CUDA;
    return SISDC_OK;
}
