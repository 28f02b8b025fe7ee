"""Element-wise fast-diagonalisation (FDS) preconditioner for the implicit
SIPG systems, FP64 (test infrastructure only).

The paper solves the implicit equations of the SI integrators by PCG or by a
fast diagonalisation solver (Sec. 8, runtime analysis) without giving the
form; the reading used here is the element-local one for the uniform
periodic mesh.  On such a mesh the SIPG stiffness is a Kronecker sum,
A = M_y (x) A_x + A_y (x) M_x with 1D line operators A_x, A_y and the 1D GLL
masses M_x = (h_x/2) W, M_y = (h_y/2) W.  Dropping the coupling to the
neighbour elements leaves, per element, the block

    B_e = M_y (x) M_x + c (M_y (x) K_x + K_y (x) M_x),

where K_x is the diagonal block of A_x belonging to one element (its volume
term and the own-element parts of both face terms).  With the generalised
eigen-decomposition K_x S_x = M_x S_x diag(lam_x), S_x^T M_x S_x = I (and the
same in y),

    B_e^{-1} = (S_y (x) S_x) diag(1 / (1 + c (lam_y[j] + lam_x[i]))) (S_y (x) S_x)^T,

i.e. four contractions of length P+1 per node (two in 1D).  It is used as
the preconditioner of CG on (M + c A) x = M b; the stopping rule is the
Jacobi one with D^{-1} replaced by B^{-1}: r^T z <= rtol^2 b^T B^{-1} b.

Pins (tests/test_oracle_fds.py): the block K_x equals the element block of
the assembled operator, B_e^{-1} applied equals a dense solve with the
element block of the assembled M + c A, and FDS-PCG reaches the dense
solution of the whole system.
"""
import numpy as np
import scipy.linalg


def element_block_1d(sp1, h):
    """Diagonal element block of the 1D periodic SIPG line operator with
    element width h, read off the operator of a 3-element line (the
    neighbours of the middle element are distinct), column by column."""
    nq = sp1.P + 1
    K = np.zeros((nq, nq))
    for k in range(nq):
        v = np.zeros((3, nq))
        v[1, k] = 1.0
        K[:, k] = sp1._sipg_line(v, h)[1, :]
    return K


class FDS:
    """The element-wise fast-diagonalisation preconditioner of one DGSpace."""

    def __init__(self, sp):
        from .dg import ConvDiff, DGSpace
        self.sp = sp
        line = DGSpace(1, (3,), sp.P, (0.0, 0.0), (3.0, 0.0), ConvDiff((0.0, 0.0), 0.0))
        self.Kx = element_block_1d(line, sp.hx)
        self.Mx = (sp.hx / 2.0) * sp.w
        self.lx, self.Sx = scipy.linalg.eigh(self.Kx, np.diag(self.Mx))
        if sp.dim == 2:
            self.Ky = element_block_1d(line, sp.hy)
            self.My = (sp.hy / 2.0) * sp.w
            self.ly, self.Sy = scipy.linalg.eigh(self.Ky, np.diag(self.My))

    def apply(self, c, r):
        """z = B^{-1} r element by element (r[c, ey, ex, j, i])."""
        Sx = self.Sx
        t = np.einsum('ai,...ja->...ji', Sx, r)                 # S_x^T along i
        if self.sp.dim == 1:
            t = t / (1.0 + c * self.lx)
            return np.einsum('ia,...ja->...ji', Sx, t)
        Sy = self.Sy
        t = np.einsum('bj,...bi->...ji', Sy, t)                 # S_y^T along j
        t = t / (1.0 + c * (self.ly[:, None] + self.lx[None, :]))
        t = np.einsum('jb,...bi->...ji', Sy, t)
        return np.einsum('ia,...ja->...ji', Sx, t)

    def block(self, c):
        """The dense element block B_e (nodes ordered j-major, i fastest)."""
        if self.sp.dim == 1:
            return np.diag(self.Mx) + c * self.Kx
        My, Mx = np.diag(self.My), np.diag(self.Mx)
        return np.kron(My, Mx) + c * (np.kron(My, self.Kx) + np.kron(self.Ky, Mx))


def pcg_fds(sp, c, rhs, x0, rtol, maxit, fds=None):
    """CG on (M + c A) x = M rhs with the FDS preconditioner; returns (x, iterations)."""
    fds = fds or FDS(sp)
    M = sp.mass
    b = M * rhs
    x = np.array(x0, dtype=float, copy=True)
    r = b - (M * x + c * sp.A(x))
    z = fds.apply(c, r)
    p = z.copy()
    rz = float(np.sum(r * z))
    bnorm2 = float(np.sum(b * fds.apply(c, b)))
    tol2 = max(rtol * rtol * bnorm2, 1e-300)
    it = 0
    while rz > tol2 and it < maxit:
        Ap = M * p + c * sp.A(p)
        alpha = rz / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        z = fds.apply(c, r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it
