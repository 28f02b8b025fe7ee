// Host tables of one level, computed in long double and rounded to double.
//
// * GLL nodes/weights and the nodal differentiation matrix on [-1, 1]
//   (DG-SEM basis, Sec. 6).
// * Collocation nodes on [0, 1] (Sec. 3.1): Radau-Right = roots of
//   P_{M-1}(x) - P_M(x) mapped by (x+1)/2; Lobatto = GLL with M points.
// * Node-to-node weights w^nn_{m,i} = int_{tau_{m-1}}^{tau_m} l_i (Sec. 3.2),
//   by M-point Gauss-Legendre quadrature per subinterval (exact).
// * Lagrange evaluation matrices for the embedded transfers (Sec. 4.2).
#include "tables.h"

#include <algorithm>
#include <cmath>

namespace sisdc {

typedef long double ld;

// P_n(x) and P_n'(x) by the three-term recurrence.
static void legendre(int n, ld x, ld* p, ld* dp) {
    ld p0 = 1.0L, p1 = x;
    if (n == 0) { *p = 1.0L; *dp = 0.0L; return; }
    for (int k = 2; k <= n; ++k) {
        const ld pk = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    *p = p1;
    // derivative from n (x P_n - P_{n-1}) / (x^2 - 1), endpoints n(n+1)/2 (+-)
    if (fabsl(fabsl(x) - 1.0L) < 1e-30L) {
        *dp = (x > 0 ? 1.0L : ((n % 2) ? 1.0L : -1.0L)) * n * (n + 1) / 2.0L;
    } else {
        *dp = n * (x * p1 - p0) / (x * x - 1.0L);
    }
}

static std::vector<ld> gauss_legendre(int n, std::vector<ld>* w) {
    std::vector<ld> x(n);
    w->assign(n, 0.0L);
    const ld pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < n; ++k) {
        ld t = cosl(pi * (k + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 100; ++it) {
            ld p, dp;
            legendre(n, t, &p, &dp);
            const ld d = p / dp;
            t -= d;
            if (fabsl(d) < 1e-19L) break;
        }
        ld p, dp;
        legendre(n, t, &p, &dp);
        x[k] = t;
        (*w)[k] = 2.0L / ((1.0L - t * t) * dp * dp);
    }
    std::vector<size_t> ord(n);
    for (int k = 0; k < n; ++k) ord[k] = k;
    std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return x[a] < x[b]; });
    std::vector<ld> xs(n), ws(n);
    for (int k = 0; k < n; ++k) { xs[k] = x[ord[k]]; ws[k] = (*w)[ord[k]]; }
    *w = ws;
    return xs;
}

static void gll_ld(int P, std::vector<ld>* x, std::vector<ld>* w) {
    x->assign(P + 1, 0.0L);
    w->assign(P + 1, 0.0L);
    const ld pi = 3.14159265358979323846264338327950288L;
    (*x)[0] = -1.0L;
    (*x)[P] = 1.0L;
    for (int k = 1; k < P; ++k) {
        // roots of P_P'(x); P_P'' from the Legendre equation
        ld t = -cosl(pi * k / P);
        for (int it = 0; it < 100; ++it) {
            ld p, dp;
            legendre(P, t, &p, &dp);
            const ld d2 = (2.0L * t * dp - P * (P + 1) * p) / (1.0L - t * t);
            const ld d = dp / d2;
            t -= d;
            if (fabsl(d) < 1e-19L) break;
        }
        (*x)[k] = t;
    }
    for (int k = 0; k <= P; ++k) {
        ld p, dp;
        legendre(P, (*x)[k], &p, &dp);
        (*w)[k] = 2.0L / (P * (P + 1) * p * p);
    }
}

static std::vector<ld> radau_right_ld(int M) {
    // roots of r(x) = P_{M-1}(x) - P_M(x) on [-1, 1]; x = 1 is one of them
    std::vector<ld> x(M);
    const ld pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < M; ++k) {
        ld t = cosl(2.0L * pi * k / (2 * M - 1));
        if (k == 0) { x[k] = 1.0L; continue; }
        for (int it = 0; it < 200; ++it) {
            ld a, da, b, db;
            legendre(M - 1, t, &a, &da);
            legendre(M, t, &b, &db);
            const ld d = (a - b) / (da - db);
            t -= d;
            if (fabsl(d) < 1e-19L) break;
        }
        x[k] = t;
    }
    std::sort(x.begin(), x.end());
    x[M - 1] = 1.0L;
    for (int k = 0; k < M; ++k) x[k] = (x[k] + 1.0L) / 2.0L;
    return x;
}

static ld lagrange(const std::vector<ld>& nodes, int j, ld t) {
    ld v = 1.0L;
    for (size_t k = 0; k < nodes.size(); ++k)
        if ((int)k != j) v *= (t - nodes[k]) / (nodes[j] - nodes[k]);
    return v;
}

std::vector<double> lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& pts) {
    std::vector<ld> nl(nodes.begin(), nodes.end());
    std::vector<double> E(pts.size() * nodes.size());
    for (size_t p = 0; p < pts.size(); ++p)
        for (size_t j = 0; j < nodes.size(); ++j)
            E[p * nodes.size() + j] = (double)lagrange(nl, (int)j, (ld)pts[p]);
    return E;
}

std::vector<double> l2_projection_matrix(int Pf, int Pc) {
    std::vector<ld> xf, wf, xc, wc;
    gll_ld(Pf, &xf, &wf);
    gll_ld(Pc, &xc, &wc);
    const int nf = Pf + 1, nc = Pc + 1;
    std::vector<ld> I(nf * nc);                        // I[k][a] = l^c_a(xf_k)
    for (int k = 0; k < nf; ++k)
        for (int a = 0; a < nc; ++a) I[k * nc + a] = lagrange(xc, a, xf[k]);
    // A = I^T W_f I (nc x nc), B = I^T W_f (nc x nf); solve A X = B
    std::vector<ld> A(nc * nc, 0.0L), B(nc * nf, 0.0L);
    for (int a = 0; a < nc; ++a) {
        for (int b = 0; b < nc; ++b)
            for (int k = 0; k < nf; ++k) A[a * nc + b] += I[k * nc + a] * wf[k] * I[k * nc + b];
        for (int k = 0; k < nf; ++k) B[a * nf + k] = I[k * nc + a] * wf[k];
    }
    for (int col = 0; col < nc; ++col) {               // Gaussian elimination, partial pivoting
        int piv = col;
        for (int r = col + 1; r < nc; ++r)
            if (fabsl(A[r * nc + col]) > fabsl(A[piv * nc + col])) piv = r;
        if (piv != col) {
            for (int q = 0; q < nc; ++q) std::swap(A[col * nc + q], A[piv * nc + q]);
            for (int q = 0; q < nf; ++q) std::swap(B[col * nf + q], B[piv * nf + q]);
        }
        for (int r = 0; r < nc; ++r) {
            if (r == col) continue;
            const ld f = A[r * nc + col] / A[col * nc + col];
            for (int q = 0; q < nc; ++q) A[r * nc + q] -= f * A[col * nc + q];
            for (int q = 0; q < nf; ++q) B[r * nf + q] -= f * B[col * nf + q];
        }
    }
    std::vector<double> P(nc * nf);
    for (int a = 0; a < nc; ++a)
        for (int k = 0; k < nf; ++k) P[a * nf + k] = (double)(B[a * nf + k] / A[a * nc + a]);
    return P;
}

void h_transfer_matrices(int Pf, int Pc, int l2, std::vector<double>* I2, std::vector<double>* P2,
                         std::vector<double>* R2) {
    std::vector<ld> xf, wf, xc, wc;
    gll_ld(Pf, &xf, &wf);
    gll_ld(Pc, &xc, &wc);
    const int nf = Pf + 1, nc = Pc + 1;
    // child c covers xi in [c - 1, c] of the coarse element: xi = (eta + 2c - 1) / 2
    std::vector<ld> I(2 * nf * nc);
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < nf; ++k)
            for (int a = 0; a < nc; ++a) I[(c * nf + k) * nc + a] = lagrange(xc, a, (xf[k] + 2 * c - 1) / 2.0L);
    I2->assign(I.begin(), I.end());
    // R = W_c^{-1} I^T W_f with the child's half width: R[c][a][k] = I[c][k][a] (wf_k / 2) / wc_a
    R2->assign(2 * nc * nf, 0.0);
    for (int c = 0; c < 2; ++c)
        for (int a = 0; a < nc; ++a)
            for (int k = 0; k < nf; ++k)
                (*R2)[(c * nc + a) * nf + k] = (double)(I[(c * nf + k) * nc + a] * (wf[k] / 2.0L) / wc[a]);
    std::vector<ld> P(2 * nc * nf, 0.0L);
    if (l2) {
        // least squares over both children: (E^T W E)^{-1} E^T W, E = [I_0; I_1], W = wf / 2
        std::vector<ld> A(nc * nc, 0.0L), B(nc * 2 * nf, 0.0L);
        for (int a = 0; a < nc; ++a) {
            for (int b = 0; b < nc; ++b)
                for (int r = 0; r < 2 * nf; ++r) A[a * nc + b] += I[r * nc + a] * (wf[r % nf] / 2.0L) * I[r * nc + b];
            for (int r = 0; r < 2 * nf; ++r) B[a * 2 * nf + r] = I[r * nc + a] * (wf[r % nf] / 2.0L);
        }
        for (int col = 0; col < nc; ++col) {           // Gauss-Jordan, partial pivoting
            int piv = col;
            for (int r = col + 1; r < nc; ++r)
                if (fabsl(A[r * nc + col]) > fabsl(A[piv * nc + col])) piv = r;
            if (piv != col) {
                for (int q = 0; q < nc; ++q) std::swap(A[col * nc + q], A[piv * nc + q]);
                for (int q = 0; q < 2 * nf; ++q) std::swap(B[col * 2 * nf + q], B[piv * 2 * nf + q]);
            }
            for (int r = 0; r < nc; ++r) {
                if (r == col) continue;
                const ld f = A[r * nc + col] / A[col * nc + col];
                for (int q = 0; q < nc; ++q) A[r * nc + q] -= f * A[col * nc + q];
                for (int q = 0; q < 2 * nf; ++q) B[r * 2 * nf + q] -= f * B[col * 2 * nf + q];
            }
        }
        for (int c = 0; c < 2; ++c)
            for (int a = 0; a < nc; ++a)
                for (int k = 0; k < nf; ++k) P[(c * nc + a) * nf + k] = B[a * 2 * nf + c * nf + k] / A[a * nc + a];
    } else {
        // embedded interpolation after linear blending: the coarse node xi takes
        // the blended left child at eta = 2 xi + 1 (xi <= 0) or the blended right
        // child at eta = 2 xi - 1; blending moves both interface values to their
        // mean with a linear ramp that vanishes at the child's outer end
        for (int a = 0; a < nc; ++a) {
            const ld xi = xc[a];
            if (xi <= 0.0L) {
                const ld eta = 2.0L * xi + 1.0L, ramp = (1.0L + eta) / 4.0L;
                for (int k = 0; k < nf; ++k) P[(0 * nc + a) * nf + k] = lagrange(xf, k, eta);
                P[(0 * nc + a) * nf + (nf - 1)] -= ramp;
                P[(1 * nc + a) * nf + 0] += ramp;
            } else {
                const ld eta = 2.0L * xi - 1.0L, ramp = (1.0L - eta) / 4.0L;
                for (int k = 0; k < nf; ++k) P[(1 * nc + a) * nf + k] = lagrange(xf, k, eta);
                P[(1 * nc + a) * nf + 0] -= ramp;
                P[(0 * nc + a) * nf + (nf - 1)] += ramp;
            }
        }
    }
    P2->assign(P.begin(), P.end());
}

bool build_level_tables(int P, int M, int lobatto, LevelTables* t) {
    if (P < 1 || P > 15 || M < 1 || M > 8 || (lobatto && M < 2)) return false;
    const int nq = P + 1;
    std::vector<ld> x, w;
    gll_ld(P, &x, &w);
    t->gll.assign(x.begin(), x.end());
    t->w.assign(w.begin(), w.end());
    // barycentric differentiation matrix
    std::vector<ld> lam(nq, 1.0L);
    for (int j = 0; j < nq; ++j)
        for (int k = 0; k < nq; ++k)
            if (k != j) lam[j] /= (x[j] - x[k]);
    t->D.assign(nq * nq, 0.0);
    std::vector<ld> Dl(nq * nq, 0.0L);
    for (int i = 0; i < nq; ++i) {
        ld diag = 0.0L;
        for (int j = 0; j < nq; ++j) {
            if (i == j) continue;
            Dl[i * nq + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            diag -= Dl[i * nq + j];
        }
        Dl[i * nq + i] = diag;
    }
    for (int k = 0; k < nq * nq; ++k) t->D[k] = (double)Dl[k];
    // K = D^T W D
    t->K.assign(nq * nq, 0.0);
    for (int i = 0; i < nq; ++i)
        for (int k = 0; k < nq; ++k) {
            ld s = 0.0L;
            for (int q = 0; q < nq; ++q) s += Dl[q * nq + i] * w[q] * Dl[q * nq + k];
            t->K[i * nq + k] = (double)s;
        }
    // diagonal of the 1D SIPG line operator on the reference scaling:
    // dline(h)[i] = (2/h) K_ii + face terms; stored as the h-independent
    // pieces, combined in level_geometry.
    t->Kdiag.resize(nq);
    for (int i = 0; i < nq; ++i) t->Kdiag[i] = t->K[i * nq + i];
    t->D00 = (double)Dl[0];
    t->DPP = (double)Dl[nq * nq - 1];
    // collocation nodes
    std::vector<ld> tau;
    if (lobatto) {
        std::vector<ld> xl, wl;
        gll_ld(M - 1, &xl, &wl);
        tau.resize(M);
        for (int k = 0; k < M; ++k) tau[k] = (xl[k] + 1.0L) / 2.0L;
        tau[0] = 0.0L;
        tau[M - 1] = 1.0L;
    } else {
        tau = radau_right_ld(M);
    }
    t->tau.assign(tau.begin(), tau.end());
    t->dtau.resize(M);
    for (int m = 0; m < M; ++m) t->dtau[m] = (double)(tau[m] - (m ? tau[m - 1] : 0.0L));
    // w^nn by Gauss-Legendre per subinterval
    std::vector<ld> gw;
    std::vector<ld> gx = gauss_legendre(M, &gw);
    t->wnn.assign(M * M, 0.0);
    for (int m = 0; m < M; ++m) {
        const ld a = m ? tau[m - 1] : 0.0L, b = tau[m];
        for (int i = 0; i < M; ++i) {
            ld s = 0.0L;
            for (int q = 0; q < M; ++q) s += gw[q] * lagrange(tau, i, a + (b - a) * (gx[q] + 1.0L) / 2.0L);
            t->wnn[m * M + i] = (double)((b - a) / 2.0L * s);
        }
    }
    return true;
}

}  // namespace sisdc

namespace sisdc {

bool gll_tables_fixed(int P, double* xo, double* wo, double* Do, double* Ko) {
    if (P < 1 || P > 8) return false;
    const int nq = P + 1;
    const ld pi = 3.14159265358979323846264338327950288L;
    ld x[9], w[9], lam[9], Dl[81];
    x[0] = -1.0L;
    x[P] = 1.0L;
    for (int k = 1; k < P; ++k) {
        ld t = -cosl(pi * k / P);
        for (int it = 0; it < 100; ++it) {
            ld p, dp;
            legendre(P, t, &p, &dp);
            const ld d = dp / ((2.0L * t * dp - P * (P + 1) * p) / (1.0L - t * t));
            t -= d;
            if (fabsl(d) < 1e-19L) break;
        }
        x[k] = t;
    }
    for (int k = 0; k < nq; ++k) {
        ld p, dp;
        legendre(P, x[k], &p, &dp);
        w[k] = 2.0L / (P * (P + 1) * p * p);
        lam[k] = 1.0L;
    }
    for (int j = 0; j < nq; ++j)
        for (int k = 0; k < nq; ++k)
            if (k != j) lam[j] /= (x[j] - x[k]);
    for (int i = 0; i < nq; ++i) {
        ld diag = 0.0L;
        for (int j = 0; j < nq; ++j) {
            if (i == j) continue;
            Dl[i * nq + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            diag -= Dl[i * nq + j];
        }
        Dl[i * nq + i] = diag;
    }
    for (int i = 0; i < nq; ++i) {
        xo[i] = (double)x[i];
        wo[i] = (double)w[i];
        for (int k = 0; k < nq; ++k) {
            Do[i * nq + k] = (double)Dl[i * nq + k];
            ld s = 0.0L;
            for (int q = 0; q < nq; ++q) s += Dl[q * nq + i] * w[q] * Dl[q * nq + k];
            Ko[i * nq + k] = (double)s;
        }
    }
    return true;
}

}  // namespace sisdc

namespace sisdc {

// Element-wise fast diagonalisation of the 1D SIPG line operator of element
// width h (the implicit systems' separable preconditioner).  The element's
// diagonal block of the line operator,
//   Kt = (2/h) D^T W D - (1/h) (e_P d_P^T + d_P e_P^T) + (1/h) (e_0 d_0^T + d_0 e_0^T)
//        + tau (e_0 e_0^T + e_P e_P^T),   d_0, d_P = first / last row of D,
//   tau = 2 (P+1)^2 / h,
// and the GLL mass Mh = (h/2) W give the generalised eigenpairs
// Kt s_i = lam_i Mh s_i with s_i^T Mh s_i = 1, found from the symmetric
// matrix Mh^{-1/2} Kt Mh^{-1/2} by cyclic Jacobi rotations (Golub & Van Loan,
// the symmetric Jacobi eigenvalue method), in long double.  Output:
// S[a * (P+1) + i] = component a of s_i, lam[i]; eigenvalues ascending.
bool fds_tables(int P, double h, double* S, double* lam) {
    if (P < 1 || P > 15 || !(h > 0.0)) return false;
    const int nq = P + 1;
    std::vector<ld> x, w;
    gll_ld(P, &x, &w);
    std::vector<ld> bl(nq, 1.0L), Dl(nq * nq, 0.0L);
    for (int j = 0; j < nq; ++j)
        for (int k = 0; k < nq; ++k)
            if (k != j) bl[j] /= (x[j] - x[k]);
    for (int i = 0; i < nq; ++i) {
        ld diag = 0.0L;
        for (int j = 0; j < nq; ++j) {
            if (i == j) continue;
            Dl[i * nq + j] = (bl[j] / bl[i]) / (x[i] - x[j]);
            diag -= Dl[i * nq + j];
        }
        Dl[i * nq + i] = diag;
    }
    const ld hl = h, tau = 2.0L * nq * nq / hl;
    std::vector<ld> C(nq * nq), V(nq * nq, 0.0L), ms(nq);
    for (int i = 0; i < nq; ++i) ms[i] = 1.0L / sqrtl(0.5L * hl * w[i]);
    for (int i = 0; i < nq; ++i)
        for (int k = 0; k < nq; ++k) {
            ld s = 0.0L;
            for (int q = 0; q < nq; ++q) s += Dl[q * nq + i] * w[q] * Dl[q * nq + k];
            s *= 2.0L / hl;
            if (k == P) s -= Dl[P * nq + i] / hl;
            if (i == P) s -= Dl[P * nq + k] / hl;
            if (k == 0) s += Dl[i] / hl;
            if (i == 0) s += Dl[k] / hl;
            if (i == k && (i == 0 || i == P)) s += tau;
            C[i * nq + k] = ms[i] * s * ms[k];
        }
    for (int i = 0; i < nq; ++i) V[i * nq + i] = 1.0L;
    for (int sweep = 0; sweep < 100; ++sweep) {
        ld off = 0.0L, tot = 0.0L;
        for (int p = 0; p < nq; ++p)
            for (int q = 0; q < nq; ++q) {
                tot += C[p * nq + q] * C[p * nq + q];
                if (p != q) off += C[p * nq + q] * C[p * nq + q];
            }
        if (off <= 1e-36L * tot) break;
        for (int p = 0; p < nq - 1; ++p)
            for (int q = p + 1; q < nq; ++q) {
                const ld apq = C[p * nq + q];
                if (apq == 0.0L) continue;
                const ld theta = (C[q * nq + q] - C[p * nq + p]) / (2.0L * apq);
                const ld t = (theta >= 0.0L ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
                const ld cs = 1.0L / sqrtl(t * t + 1.0L), sn = t * cs;
                for (int k = 0; k < nq; ++k) {          // columns p, q
                    const ld ckp = C[k * nq + p], ckq = C[k * nq + q];
                    C[k * nq + p] = cs * ckp - sn * ckq;
                    C[k * nq + q] = sn * ckp + cs * ckq;
                }
                for (int k = 0; k < nq; ++k) {          // rows p, q
                    const ld cpk = C[p * nq + k], cqk = C[q * nq + k];
                    C[p * nq + k] = cs * cpk - sn * cqk;
                    C[q * nq + k] = sn * cpk + cs * cqk;
                }
                for (int k = 0; k < nq; ++k) {
                    const ld vkp = V[k * nq + p], vkq = V[k * nq + q];
                    V[k * nq + p] = cs * vkp - sn * vkq;
                    V[k * nq + q] = sn * vkp + cs * vkq;
                }
            }
    }
    std::vector<int> order(nq);
    for (int i = 0; i < nq; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return C[a * nq + a] < C[b * nq + b]; });
    for (int i = 0; i < nq; ++i) {
        const int o = order[i];
        lam[i] = (double)C[o * nq + o];
        for (int a = 0; a < nq; ++a) S[a * nq + i] = (double)(ms[a] * V[a * nq + o]);
    }
    return true;
}

}  // namespace sisdc


namespace sisdc {

// Nodal-to-modal matrix of the artificial-viscosity sensor: the inverse of
// V[i][k] = sqrt((2k+1)/2) P_k(x_i) on the GLL nodes x_i (orthonormal
// Legendre modes), by Gauss-Jordan elimination with partial pivoting in long
// double.  out[k * (P+1) + i]: coefficient of mode k from nodal value i.
bool modal_matrix(int P, double* out) {
    const int n = P + 1;
    std::vector<ld> x, w;
    gll_ld(P, &x, &w);
    std::vector<ld> A(n * 2 * n, 0.0L);      // [V | I]
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < n; ++k) {
            ld p, dp;
            legendre(k, x[i], &p, &dp);
            A[i * 2 * n + k] = sqrtl((2.0L * k + 1.0L) / 2.0L) * p;
        }
        A[i * 2 * n + n + i] = 1.0L;
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * 2 * n + c]) > fabsl(A[piv * 2 * n + c])) piv = r;
        if (fabsl(A[piv * 2 * n + c]) < 1e-30L) return false;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) std::swap(A[c * 2 * n + k], A[piv * 2 * n + k]);
        const ld d = A[c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) A[c * 2 * n + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const ld f = A[r * 2 * n + c];
            if (f == 0.0L) continue;
            for (int k = 0; k < 2 * n; ++k) A[r * 2 * n + k] -= f * A[c * 2 * n + k];
        }
    }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) out[k * n + i] = (double)A[k * 2 * n + n + i];
    return true;
}

}  // namespace sisdc
