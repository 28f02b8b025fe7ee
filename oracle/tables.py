"""Collocation and spectral-element tables in FP64 (test infrastructure only).

* Collocation nodes on [0, 1] (Sec. 3.1): Radau-Right (t_1 > t_0, t_M = 1)
  and Lobatto (t_1 = t_0 = 0, t_M = 1).
* Node-to-node weights w^nn_{m,i} = int_{tau_{m-1}}^{tau_m} l_i(tau) dtau
  (Sec. 3.2, eq. nn_weights) with tau_0 = 0 and l_i the Lagrange basis on
  tau_1..tau_M; zero-to-node weights w^0n = cumulative sum (Sec. 3.4,
  eq. 0n_weights).
* GLL nodes, weights and the nodal differentiation matrix on [-1, 1] for the
  DG-SEM space of Sec. 6.
* Lagrange evaluation matrices used for the embedded interpolation
  transfers of Sec. 4.2 and Sec. 6.2.

Pins (tests/test_oracle_tables.py): cumulative weights equal the textbook
Radau IIA / Lobatto IIIA Butcher matrices, the printed 3x4 matrices of
Sec. 4.6, quadrature exactness, D exact on polynomials of degree <= P.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def _legendre_coeffs(n):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return c


def _newton_polish(f, df, x, iters=3):
    for _ in range(iters):
        x = x - f(x) / df(x)
    return x


def gll(P):
    """GLL nodes x (ascending) and weights w on [-1, 1] for degree P >= 1.

    Nodes: the endpoints and the roots of P_P'(x); weights
    w_i = 2 / (P (P+1) P_P(x_i)^2)."""
    if P < 1:
        raise ValueError("P >= 1 required")
    cP = _legendre_coeffs(P)
    d1 = npleg.legder(cP)
    d2 = npleg.legder(d1)
    interior = np.sort(np.real(npleg.legroots(d1))) if P >= 2 else np.zeros(0)
    if P >= 2:
        interior = _newton_polish(lambda t: npleg.legval(t, d1),
                                  lambda t: npleg.legval(t, d2), interior)
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (P * (P + 1) * npleg.legval(x, cP) ** 2)
    return x, w


def barycentric_weights(x):
    n = len(x)
    lam = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                lam[j] /= (x[j] - x[k])
    return lam


def diff_matrix(x):
    """Nodal differentiation matrix D_ij = l_j'(x_i) (barycentric form)."""
    n = len(x)
    lam = barycentric_weights(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def lagrange_matrix(nodes, points):
    """E[p, j] = l_j(points[p]) for the Lagrange basis on ``nodes``
    (plain product formula)."""
    nodes = np.asarray(nodes, dtype=float)
    points = np.asarray(points, dtype=float)
    E = np.ones((len(points), len(nodes)))
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                E[:, j] *= (points - nodes[k]) / (nodes[j] - nodes[k])
    return E


def radau_right(M):
    """Radau-Right collocation nodes on [0, 1] (includes 1, excludes 0):
    roots of P_{M-1}(x) - P_M(x) on [-1, 1], mapped by (x + 1) / 2."""
    if M < 1:
        raise ValueError("M >= 1 required")
    c = np.zeros(M + 1)
    c[M - 1] += 1.0
    c[M] -= 1.0
    r = np.sort(np.real(npleg.legroots(c)))
    dc = npleg.legder(c)
    r = _newton_polish(lambda t: npleg.legval(t, c), lambda t: npleg.legval(t, dc), r)
    r[-1] = 1.0
    return (r + 1.0) / 2.0


def lobatto(M):
    """Lobatto collocation nodes on [0, 1] (includes both endpoints)."""
    if M < 2:
        raise ValueError("M >= 2 required for Lobatto nodes")
    x, _ = gll(M - 1)
    t = (x + 1.0) / 2.0
    t[0], t[-1] = 0.0, 1.0
    return t


def collocation_nodes(kind, M):
    if kind == "radau_right":
        return radau_right(M)
    if kind == "lobatto":
        return lobatto(M)
    raise ValueError(kind)


def wnn(tau):
    """w^nn[m-1, i-1] = int_{tau_{m-1}}^{tau_m} l_i(s) ds on the unit interval,
    tau_0 = 0 (Sec. 3.2).  Gauss-Legendre with M points per subinterval is
    exact for the degree M-1 integrand."""
    tau = np.asarray(tau, dtype=float)
    M = len(tau)
    gx, gw = npleg.leggauss(M)
    W = np.zeros((M, M))
    prev = 0.0
    for m in range(M):
        a, b = prev, tau[m]
        s = a + (b - a) * (gx + 1.0) / 2.0
        L = lagrange_matrix(tau, s)          # (ng, M)
        W[m, :] = (b - a) / 2.0 * (gw @ L)
        prev = tau[m]
    return W


def w0n(tau):
    """Zero-to-node weights w^0n_{m,i} = sum_{j<=m} w^nn_{j,i} (Sec. 3.4)."""
    return np.cumsum(wnn(tau), axis=0)


def substeps(tau):
    """Delta t_m / Delta t = tau_m - tau_{m-1}, tau_0 = 0."""
    tau = np.asarray(tau, dtype=float)
    return np.diff(np.concatenate([[0.0], tau]))


def c0n(M):
    """C^0n: lower-triangular matrix of ones (Sec. 4.5)."""
    return np.tril(np.ones((M, M)))


def time_transfers(tau_f, tau_c):
    """Embedded time transfers between collocation node sets (Sec. 4.2).

    I_t (M_f x M_c): coarse Lagrange interpolant (on tau^c_1..tau^c_Mc, t_0
    excluded) evaluated at the fine nodes.  P_t (M_c x M_f): fine interpolant
    evaluated at the coarse nodes.  R_t = I_t^T (eq. restriction)."""
    It = lagrange_matrix(tau_c, tau_f)
    Pt = lagrange_matrix(tau_f, tau_c)
    return It, Pt, It.T.copy()


def space_transfers(P_f, P_c):
    """Per-direction p-coarsening transfers on one element (Sec. 6.2).

    I_x ((P_f+1) x (P_c+1)): coarse GLL Lagrange basis at the fine GLL nodes
    (embedded interpolation).  P_x ((P_c+1) x (P_f+1)): fine polynomial at
    the coarse GLL nodes.  R_x = W_c^{-1} I_x^T W_f: the transpose of I_x in
    the GLL-mass inner product, so nodal residuals restrict as mass-weighted
    vectors (reading: the weak form makes residuals mass-weighted)."""
    xf, wf = gll(P_f)
    xc, wc = gll(P_c)
    Ix = lagrange_matrix(xc, xf)
    Px = lagrange_matrix(xf, xc)
    Rx = (Ix.T * wf[None, :]) / wc[:, None]
    return Ix, Px, Rx


def l2_projection(P_f, P_c):
    """Per-direction L2 projection of a degree-P_f element polynomial onto
    degree P_c (the alternative solution projection of Sec. 4.2), with the
    inner product of the fine GLL quadrature: the coarse coefficients c
    minimise sum_k wf_k (u_k - (I_x c)_k)^2, i.e.
    P = (I_x^T W_f I_x)^{-1} I_x^T W_f (the coarse mass here is the consistent
    one, exact for degree 2 P_c <= 2 P_f - 1)."""
    xf, wf = gll(P_f)
    xc, _ = gll(P_c)
    Ix = lagrange_matrix(xc, xf)
    Mc = Ix.T @ (wf[:, None] * Ix)
    return np.linalg.solve(Mc, Ix.T * wf[None, :])


def h_transfers(P_f, P_c, projection="interp"):
    """Per-direction transfers for 2:1 h-coarsening (Sec. 6.2: two adjacent
    fine elements fused into one coarse element), optionally with p-coarsening.
    Fine child c (0 = left, 1 = right) covers the half [-1, 0] or [0, 1] of
    the coarse reference element: coarse coordinate xi = (eta - 1) / 2 or
    (eta + 1) / 2 of the child's coordinate eta.

    Returns lists over the two children:
    I[c] ((P_f+1) x (P_c+1)): the coarse polynomial evaluated at the child's
        GLL nodes (exact for coarse polynomials);
    P[c] ((P_c+1) x (P_f+1)): the solution projection, as the contribution of
        child c's nodal values to the coarse nodal values.  "interp"
        (default): embedded interpolation after removing the jump between the
        two children by linear blending -- each child is corrected by a linear
        function that vanishes at its outer end so that both meet the mean of
        their two interface values -- then each coarse node takes the value
        of the child whose half contains it (the centre node, where both
        agree, takes their mean).  "l2": the least-squares fit over both
        children under the fine GLL quadrature (no blending);
    R[c] ((P_c+1) x (P_f+1)): the residual restriction R = W_c^{-1} I^T W_f
        with the masses of the two widths (the child is half as wide), the
        transpose of I in the mass inner product.

    Readings (the paper names the blending but not its form): linear
    blending as above; the tensor product of these 1D maps in 2D.  Each map
    is built here from its definition applied to unit vectors."""
    xf, wf = gll(P_f)
    xc, wc = gll(P_c)
    nf, nc = P_f + 1, P_c + 1
    I = [lagrange_matrix(xc, (xf - 1.0) / 2.0), lagrange_matrix(xc, (xf + 1.0) / 2.0)]
    R = [(I[c].T * (0.5 * wf)[None, :]) / wc[:, None] for c in range(2)]

    def blended_value(uL, uR, xi):
        """Value at coarse coordinate xi of the blended two-child function."""
        mean = 0.5 * (uL[-1] + uR[0])
        if xi <= 0.0:
            eta = 2.0 * xi + 1.0
            base = float(lagrange_matrix(xf, np.array([eta]))[0] @ uL)
            return base + (mean - uL[-1]) * (1.0 + eta) / 2.0
        eta = 2.0 * xi - 1.0
        base = float(lagrange_matrix(xf, np.array([eta]))[0] @ uR)
        return base + (mean - uR[0]) * (1.0 - eta) / 2.0

    P = [np.zeros((nc, nf)), np.zeros((nc, nf))]
    if projection == "l2":
        E = np.vstack(I)                                   # (2 nf) x nc
        W = np.concatenate([0.5 * wf, 0.5 * wf])
        Pl = np.linalg.solve(E.T @ (W[:, None] * E), E.T * W[None, :])
        P = [Pl[:, :nf], Pl[:, nf:]]
    else:
        for c in range(2):
            for b in range(nf):
                u = [np.zeros(nf), np.zeros(nf)]
                u[c][b] = 1.0
                for a in range(nc):
                    P[c][a, b] = blended_value(u[0], u[1], xc[a])
    return I, P, R
