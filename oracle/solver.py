"""Jacobi-preconditioned conjugate gradients in FP64 (test infrastructure only).

The implicit equations of the SI integrators are solved "to convergence"
by preconditioned CG (Sec. 8, runtime analysis).  The preconditioner is
not stated; the reading used on both sides is Jacobi (the diagonal of
M + c A).  Stopping rule: r^T z <= rtol^2 * b^T D^{-1} b (the
preconditioned residual norm relative to that of the right-hand side),
at most ``maxit`` iterations.
"""
import numpy as np


def pcg(apply_op, diag, b, x0, rtol, maxit):
    x = np.array(x0, dtype=float, copy=True)
    r = b - apply_op(x)
    z = r / diag
    p = z.copy()
    rz = float(np.sum(r * z))
    bnorm2 = float(np.sum(b * b / diag))
    tol2 = max(rtol * rtol * bnorm2, 1e-300)
    it = 0
    while rz > tol2 and it < maxit:
        Ap = apply_op(p)
        alpha = rz / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        z = r / diag
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it
