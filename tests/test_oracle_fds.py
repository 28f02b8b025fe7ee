"""Pins for the oracle's element-wise fast-diagonalisation preconditioner
(CPU only): its element block is the diagonal block of the assembled SIPG
operator, its application is a dense solve with that block, and CG with it
reaches the dense solution of the whole implicit system (Sec. 8 runs the
implicit solves with PCG or a fast diagonalisation solver)."""
import numpy as np
import pytest

from oracle.dg import Burgers2, ConvDiff, DGSpace
from oracle.fds import FDS, pcg_fds


def _dense(sp, op):
    n = int(np.prod(sp.shape))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = op(e.reshape(sp.shape)).ravel()
    return A


def _elem_index(sp, ey, ex):
    """Flat indices (component 0) of the nodes of element (ey, ex), j-major."""
    idx = np.arange(int(np.prod(sp.shape))).reshape(sp.shape)
    return idx[0, ey, ex].ravel()


@pytest.mark.parametrize("dim,nel,P", [(1, (4,), 4), (2, (3, 4), 3), (2, (4, 3), 5)])
def test_element_block_is_diagonal_block_of_assembled_operator(dim, nel, P):
    sp = DGSpace(dim, nel, P, (0.0, 0.0), (1.0, 2.0), ConvDiff((1.0, 0.5), 0.01))
    c = 0.037
    B = _dense(sp, lambda v: sp.mass * v + c * sp.A(v))
    f = FDS(sp)
    Be = f.block(c)
    for ey in range(sp.ney):
        for ex in range(sp.nex):
            ii = _elem_index(sp, ey, ex)
            assert np.allclose(B[np.ix_(ii, ii)], Be, rtol=0, atol=1e-12 * np.max(np.abs(Be)))


@pytest.mark.parametrize("dim,nel,P,c", [(1, (5,), 6, 0.01), (2, (3, 3), 4, 0.002), (2, (2, 3), 7, 0.3)])
def test_apply_is_dense_element_solve(dim, nel, P, c):
    sp = DGSpace(dim, nel, P, (0.0, 0.0), (1.0, 1.5), ConvDiff((1.0, 0.5), 0.01))
    f = FDS(sp)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(sp.shape)
    z = f.apply(c, r)
    Be = f.block(c)
    for ey in range(sp.ney):
        for ex in range(sp.nex):
            want = np.linalg.solve(Be, r[0, ey, ex].ravel())
            assert np.allclose(z[0, ey, ex].ravel(), want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))
    # the eigenbasis is M-orthonormal and diagonalises K
    assert np.allclose(f.Sx.T @ np.diag(f.Mx) @ f.Sx, np.eye(P + 1), atol=1e-12)
    assert np.allclose(f.Sx.T @ f.Kx @ f.Sx, np.diag(f.lx), atol=1e-9 * np.max(np.abs(f.lx)))


@pytest.mark.parametrize("dim,nel,P,ncomp", [(1, (6,), 5, 1), (2, (3, 4), 4, 1), (2, (3, 3), 3, 2)])
def test_fds_pcg_reaches_dense_solution(dim, nel, P, ncomp):
    pde = ConvDiff((1.0, 0.5), 0.01) if ncomp == 1 else Burgers2(0.01)
    sp = DGSpace(dim, nel, P, (0.0, 0.0), (1.0, 1.0), pde)
    c = 0.02
    rng = np.random.default_rng(9)
    rhs = rng.standard_normal(sp.shape)
    B = _dense(sp, lambda v: sp.mass * v + c * sp.A(v))
    want = np.linalg.solve(B, (sp.mass * rhs).ravel()).reshape(sp.shape)
    x, it = pcg_fds(sp, c, rhs, np.zeros(sp.shape), 1e-14, 1000)
    assert np.max(np.abs(x - want)) < 1e-11 * np.max(np.abs(want))
    xj = sp.solve(c, rhs, np.zeros(sp.shape))
    assert it <= sp.last_cg_iters[-1]


def test_fds_is_exact_on_a_single_element_per_direction_without_coupling():
    """With c = 0 the preconditioner is M^{-1}: one iteration solves M x = M b."""
    sp = DGSpace(2, (3, 3), 4, (0.0, 0.0), (1.0, 1.0), ConvDiff((1.0, 0.5), 0.01))
    rng = np.random.default_rng(1)
    r = rng.standard_normal(sp.shape)
    assert np.allclose(FDS(sp).apply(0.0, r), r / sp.mass, rtol=1e-12)
