// Host tables of one level (long double construction, double storage).
#pragma once
#include <vector>

namespace sisdc {

struct LevelTables {
    std::vector<double> gll, w, D, K, Kdiag;   // GLL nodes/weights, D, D^T W D
    double D00 = 0.0, DPP = 0.0;
    std::vector<double> tau, dtau, wnn;        // collocation nodes, substeps, w^nn
};

bool build_level_tables(int P, int M, int lobatto, LevelTables* t);

// E[p][j] = l_j(pts[p]) for the Lagrange basis on `nodes`.
std::vector<double> lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& pts);

// 2:1 h-coarsening transfers per direction (children 0 = left, 1 = right half
// of the coarse element), child-major: I2 [2][(Pf+1) x (Pc+1)] coarse
// polynomial at the child's nodes; P2 [2][(Pc+1) x (Pf+1)] solution
// projection (embedded interpolation after linear blending of the jump
// between the children, or with l2 != 0 the least-squares fit over both
// children); R2 [2][(Pc+1) x (Pf+1)] = W_c^-1 I^T W_f (half-width children).
void h_transfer_matrices(int Pf, int Pc, int l2, std::vector<double>* I2, std::vector<double>* P2,
                         std::vector<double>* R2);

// Element-wise fast diagonalisation of the 1D SIPG line operator of element
// width h: S[a * (P+1) + i] = component a of the i-th generalised eigenvector
// of (element block, GLL mass), M-orthonormal; lam[i] ascending.
bool fds_tables(int P, double h, double* S, double* lam);

// Nodal-to-modal matrix of degree P (orthonormal Legendre modes on the GLL
// nodes): out[k * (P+1) + i], mode k from nodal value i.
bool modal_matrix(int P, double* out);

// Per-direction L2 projection from degree Pf to Pc under the fine GLL
// quadrature: (I^T W_f I)^{-1} I^T W_f, row-major (Pc+1) x (Pf+1).
std::vector<double> l2_projection_matrix(int Pf, int Pc);

}  // namespace sisdc

namespace sisdc {
// GLL nodes x, weights w, differentiation matrix D and K = D^T W D for degree
// P (1..8) into caller arrays of at least 9, 9, 81, 81 doubles; no heap use.
bool gll_tables_fixed(int P, double* x, double* w, double* D, double* K);
}  // namespace sisdc
