"""Pins for the oracle's 2:1 h-coarsening transfers (CPU only; Sec. 6.2,
"MLSDC transfer operators": two adjacent fine elements fused into one coarse
element, jumps removed by linear blending, R the transpose of I).

* I is exact: the coarse piecewise polynomial evaluated at the fine nodes'
  physical coordinates (computed here from the two meshes' coordinates);
* P o I = id for embedded interpolation and for the L2 projection;
* R = I^T in the GLL-mass inner products of the two meshes, and R 1 = 1;
* linear blending: across a jump the coarse centre node takes the mean of the
  two interface values, the outer nodes keep the children's outer values;
* whole method: a V-cycle started at the fine collocation solution leaves it
  unchanged (FAS fixed point), and h-coarsened MLSDC converges to the dense
  collocation solution, in 1D and 2D.
"""
import math

import numpy as np
import pytest

from oracle import sdc as S
from oracle.dg import ConvDiff, DGSpace
from oracle.mlsdc import MLSDC, Transfer
from oracle.sdc import Level
from oracle.tables import collocation_nodes, gll, lagrange_matrix, w0n


def _spaces(dim, nel_c, Pf, Pc, ry=2):
    pde = ConvDiff((1.0, 0.6), 0.03)
    hi = (2 * math.pi, 1.5)
    nc = tuple(nel_c[:dim])
    nf = (2 * nel_c[0],) + ((ry * nel_c[1],) if dim == 2 else ())
    fine = DGSpace(dim, nf, Pf, (0.0, 0.0), hi, pde, cg_rtol=1e-15)
    coarse = DGSpace(dim, nc, Pc, (0.0, 0.0), hi, pde, cg_rtol=1e-15)
    return fine, coarse


def _transfer(fine, coarse, projection="interp"):
    return Transfer(Level(fine, "radau_right", 3), Level(coarse, "radau_right", 2), projection)


def _eval_coarse_at(coarse, uc, X, Y):
    """The coarse piecewise polynomial at the fine nodes' physical points
    (X, Y)[ey, ex, j, i]; each fine element lies in the coarse element that
    contains its centre (the element's own polynomial at shared end points)."""
    xg, _ = gll(coarse.P)
    out = np.zeros((coarse.ncomp,) + X.shape)
    Xc = X.mean(axis=(2, 3))
    Yc = Y.mean(axis=(2, 3))
    for idx in np.ndindex(X.shape):
        x = X[idx]
        ex = int((Xc[idx[:2]] - coarse.lo[0]) // coarse.hx)
        xi = 2.0 * (x - coarse.lo[0] - ex * coarse.hx) / coarse.hx - 1.0
        lx = lagrange_matrix(xg, np.array([xi]))[0]
        if coarse.dim == 1:
            out[(slice(None),) + idx] = uc[:, 0, ex, 0, :] @ lx
            continue
        y = Y[idx]
        ey = int((Yc[idx[:2]] - coarse.lo[1]) // coarse.hy)
        eta = 2.0 * (y - coarse.lo[1] - ey * coarse.hy) / coarse.hy - 1.0
        ly = lagrange_matrix(xg, np.array([eta]))[0]
        out[(slice(None),) + idx] = np.einsum('cji,j,i->c', uc[:, ey, ex], ly, lx)
    return out


@pytest.mark.parametrize("dim,nel_c,Pf,Pc,ry", [(1, (3,), 4, 4, 1), (1, (4,), 6, 3, 1), (2, (2, 3), 3, 3, 2),
                                               (2, (3, 2), 5, 3, 2), (2, (2, 2), 4, 2, 1)])
def test_interpolation_is_exact(dim, nel_c, Pf, Pc, ry):
    fine, coarse = _spaces(dim, nel_c, Pf, Pc, ry)
    T = _transfer(fine, coarse)
    uc = np.random.default_rng(3).standard_normal(coarse.shape)
    X, Y = fine.coords()
    want = _eval_coarse_at(coarse, uc, X, Y)
    got = T._space('I', uc)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("projection", ["interp", "l2"])
@pytest.mark.parametrize("dim,Pf,Pc", [(1, 5, 5), (1, 7, 3), (2, 4, 4), (2, 5, 2)])
def test_projection_inverts_interpolation(projection, dim, Pf, Pc):
    fine, coarse = _spaces(dim, (3, 2), Pf, Pc)
    T = _transfer(fine, coarse, projection)
    uc = np.random.default_rng(5).standard_normal(coarse.shape)
    assert np.max(np.abs(T._space('P', T._space('I', uc)) - uc)) < 1e-12 * np.max(np.abs(uc))


@pytest.mark.parametrize("dim,Pf,Pc", [(1, 4, 4), (1, 6, 3), (2, 3, 3), (2, 5, 3)])
def test_restriction_is_mass_transpose_of_interpolation(dim, Pf, Pc):
    fine, coarse = _spaces(dim, (3, 2), Pf, Pc)
    T = _transfer(fine, coarse)
    rng = np.random.default_rng(8)
    rf = rng.standard_normal(fine.shape)
    vc = rng.standard_normal(coarse.shape)
    lhs = np.sum(coarse.mass * T._space('R', rf) * vc)
    rhs = np.sum(fine.mass * rf * T._space('I', vc))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)
    ones = T._space('R', np.ones(fine.shape))
    assert np.max(np.abs(ones - 1.0)) < 1e-13


@pytest.mark.parametrize("Pc", [4, 5])
def test_linear_blending_across_a_jump(Pc):
    """Two children with constant values a and b: the blended function is
    linear from a (left end) through (a+b)/2 (interface) to b (right end)."""
    fine, coarse = _spaces(1, (2,), 6, Pc)
    T = _transfer(fine, coarse)
    uf = np.zeros(fine.shape)
    a, b = 1.0, 3.0
    uf[0, 0, 0::2, 0, :] = a          # left children
    uf[0, 0, 1::2, 0, :] = b          # right children
    uc = T._space('P', uf)
    xc, _ = gll(Pc)
    # inside each coarse element: a + (b - a) (xi + 1)/2
    want = a + (b - a) * (xc + 1.0) / 2.0
    assert np.max(np.abs(uc[0, 0, 0, 0, :] - want)) < 1e-13
    assert np.max(np.abs(uc[0, 0, 1, 0, :] - want)) < 1e-13


def _dense_f(sp):
    n = int(np.prod(sp.shape))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = S.f_eval(sp, e.reshape(sp.shape)).ravel()
    return A


def _collocation(sp, kind, M, u0, dt):
    Ah = _dense_f(sp)
    W = w0n(collocation_nodes(kind, M))
    n = Ah.shape[0]
    U = np.linalg.solve(np.eye(M * n) - dt * np.kron(W, Ah), np.tile(u0.ravel(), M))
    return U.reshape((M,) + sp.shape)


@pytest.mark.parametrize("dim,projection", [(1, "interp"), (1, "l2"), (2, "interp")])
def test_h_coarsened_mlsdc_fixed_point_and_convergence(dim, projection):
    if dim == 1:
        fine, coarse = _spaces(1, (3,), 5, 5)
        X, _ = fine.coords()
        u0 = (np.sin(X) + 0.3 * np.cos(2 * X))[None]
        dt = 0.25
    else:
        fine, coarse = _spaces(2, (2, 2), 3, 3)
        X, Y = fine.coords()
        u0 = (np.sin(X) * np.cos(2 * math.pi * Y / 1.5))[None]
        dt = 0.1
    kind = "radau_right"
    Uc = _collocation(fine, kind, 4, u0, dt)
    ml = MLSDC([Level(coarse, kind, 3), Level(fine, kind, 4)], stages=2, projection=projection)
    u0s = ml.initial_values(u0)
    Us = [np.zeros((3,) + coarse.shape), Uc.copy()]
    ml.vcycle(u0s, Us, dt)
    assert np.max(np.abs(Us[-1] - Uc)) < 1e-12 * max(1.0, np.max(np.abs(Uc)))
    errs = []
    for nc in (1, 6, 80):
        _, L = ml.step(u0, dt, nc, start="cascade", return_levels=True)
        errs.append(np.max(np.abs(L[-1] - Uc)))
    assert errs[-1] < 1e-11 and errs[0] > errs[1] > errs[2]
