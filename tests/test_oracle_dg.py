"""Pins for the oracle's DG-SEM operators (CPU only): SIPG symmetry,
semi-definiteness and kernel; strong form == an independently written
weak form; spectral accuracy against closed-form derivatives; the exact
time derivative of the translating isentropic vortex; conservation."""
import math

import numpy as np
import pytest

from oracle.dg import DGSpace, ConvDiff, Burgers2, Euler2
from paper_2504_18526_gb300 import inputs


def dense(sp, op):
    n = int(np.prod(sp.shape))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = op(e.reshape(sp.shape)).ravel()
    return A


@pytest.mark.parametrize("dim,nel,P", [(1, (5,), 4), (1, (3,), 1), (2, (3, 4), 3),
                                       (2, (3, 3), 7), (2, (2, 3), 2)])
def test_sipg_spd_kernel_diag(dim, nel, P):
    sp = DGSpace(dim, nel, P, (0.0, 0.0), (1.0, 2.0), ConvDiff((1.0, 0.5), 0.01))
    A = dense(sp, sp.A)
    scale = np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) < 1e-13 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-12 * scale
    # kernel is exactly the constants (one zero eigenvalue on a connected mesh)
    assert np.sum(ev < 1e-10 * scale) == 1
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-12 * scale
    assert np.allclose(np.diag(A), np.broadcast_to(sp.diagA, sp.shape).ravel(), atol=1e-12 * scale)


def _weak_conv_loops(sp, u):
    """Weak form written with explicit loops:
    (h/2) w_i c_i = sum_k w_k D_ki F_k - phi_i F* |_right + phi_i F* |_left
    per grid line (the GLL mass in the other direction cancels)."""
    pde, D, w, P = sp.pde, sp.D, sp.w, sp.P
    nc, ney, nex, nqy, nqx = sp.shape
    c = np.zeros_like(u)

    def line(vals, fluxf, rhof, h):
        # vals: (ne, nc, nq) states along one line of elements
        ne = vals.shape[0]
        out = np.zeros_like(vals)
        for e in range(ne):
            F = np.stack([fluxf(vals[e][:, k:k + 1])[:, 0] for k in range(P + 1)], axis=1)
            for i in range(P + 1):
                out[e][:, i] += sum(w[k] * D[k, i] * F[:, k] for k in range(P + 1))
            uL, uR = vals[e][:, -1:], vals[(e + 1) % ne][:, :1]
            lam = max(rhof(uL)[0], rhof(uR)[0])
            Fs = 0.5 * (fluxf(uL) + fluxf(uR))[:, 0] - 0.5 * lam * (uR - uL)[:, 0]
            out[e][:, -1] -= Fs
            out[(e + 1) % ne][:, 0] += Fs
        return out * (2.0 / h) / w[None, None, :]

    for ey in range(ney):
        for j in range(nqy):
            vals = np.stack([u[:, ey, e, j, :] for e in range(nex)])
            res = line(vals, pde.flux_x, pde.rho_x, sp.hx)
            for e in range(nex):
                c[:, ey, e, j, :] += res[e]
    if sp.dim == 2:
        for ex in range(nex):
            for i in range(nqx):
                vals = np.stack([u[:, e, ex, :, i] for e in range(ney)])
                res = line(vals, pde.flux_y, pde.rho_y, sp.hy)
                for e in range(ney):
                    c[:, e, ex, :, i] += res[e]
    return c


@pytest.mark.parametrize("pdename", ["convdiff1d", "convdiff", "burgers", "euler"])
def test_strong_equals_weak(pdename):
    rng = np.random.default_rng(3)
    if pdename == "convdiff1d":
        sp = DGSpace(1, (4,), 5, (0, 0), (1, 0), ConvDiff((0.7, 0.0), 0.0))
        u = rng.standard_normal(sp.shape)
    elif pdename == "convdiff":
        sp = DGSpace(2, (3, 2), 4, (0, 0), (1, 1), ConvDiff((0.7, -1.3), 0.0))
        u = rng.standard_normal(sp.shape)
    elif pdename == "burgers":
        sp = DGSpace(2, (2, 3), 3, (0, 0), (1, 2), Burgers2(0.0))
        u = rng.standard_normal(sp.shape)
    else:
        sp = DGSpace(2, (2, 2), 3, (0, 0), (1, 1), Euler2(1.4))
        u = np.empty(sp.shape)
        u[0] = 1.0 + 0.2 * rng.random(sp.shape[1:])
        u[1] = 0.3 * rng.standard_normal(sp.shape[1:])
        u[2] = 0.3 * rng.standard_normal(sp.shape[1:])
        u[3] = 2.5 + 0.2 * rng.random(sp.shape[1:])
    strong = sp.conv(u)
    weak = _weak_conv_loops(sp, u)
    assert np.max(np.abs(strong - weak)) < 1e-11 * max(1.0, np.max(np.abs(strong)))


def test_spectral_accuracy_convdiff_and_lap():
    errs = []
    for P in (4, 7, 10):
        sp = DGSpace(2, (4, 4), P, (0, 0), (2 * math.pi, 2 * math.pi), ConvDiff((1.0, 0.5), 0.01))
        X, Y = sp.coords()
        u = np.sin(X + 2 * Y)[None]
        ce = -(1.0 + 0.5 * 2.0) * np.cos(X + 2 * Y)
        errs.append((np.max(np.abs(sp.conv(u)[0] - ce)),
                     np.max(np.abs(sp.lap(u)[0] + 5.0 * np.sin(X + 2 * Y)))))
    assert errs[-1][0] < 1e-6 and errs[-1][1] < 1e-5
    assert errs[0][0] > 100 * errs[-1][0] and errs[0][1] > 100 * errs[-1][1]


def test_burgers_flux_divergence():
    sp = DGSpace(2, (4, 4), 10, (0, 0), (1, 1), Burgers2(0.0))
    X, Y = sp.coords()
    s, c2 = np.sin, np.cos
    k = 2 * math.pi
    u1 = s(k * X) * c2(k * Y)
    u2 = -c2(k * X) * s(k * Y)
    u = np.stack([u1, u2])
    # -d_x(u1^2) - d_y(u1 u2), -d_x(u1 u2) - d_y(u2^2)
    du1x, du1y = k * c2(k * X) * c2(k * Y), -k * s(k * X) * s(k * Y)
    du2x, du2y = k * s(k * X) * s(k * Y), -k * c2(k * X) * c2(k * Y)
    e1 = -(2 * u1 * du1x) - (du1y * u2 + u1 * du2y)
    e2 = -(du1x * u2 + u1 * du2x) - (2 * u2 * du2y)
    c = sp.conv(u)
    assert np.max(np.abs(c[0] - e1)) < 1e-5 and np.max(np.abs(c[1] - e2)) < 1e-5


def test_euler_vortex_time_derivative():
    """For the exactly translating vortex, c(u) = -div F(u) = du/dt."""
    errs = []
    for P in (6, 12):
        sp = DGSpace(2, (16, 16), P, (-10, -10), (10, 10), Euler2(1.4))
        X, Y = sp.coords()
        d = 1e-4
        dudt = (inputs.isentropic_vortex(X, Y, d) - inputs.isentropic_vortex(X, Y, -d)) / (2 * d)
        u = inputs.isentropic_vortex(X, Y, 0.0)
        errs.append(np.max(np.abs(sp.conv(u) - dudt)))
    assert errs[1] < 1e-5 and errs[0] > 10 * errs[1]


@pytest.mark.parametrize("pde", [ConvDiff((1.0, -0.5), 0.1), Burgers2(0.1), Euler2(1.4)])
def test_conservation_and_freestream(pde):
    sp = DGSpace(2, (3, 4), 4, (0, 0), (1, 2), pde)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(sp.shape)
    if isinstance(pde, Euler2):
        u[0] = 1 + 0.1 * np.abs(u[0])
        u[1:3] *= 0.3
        u[3] = 3 + 0.1 * np.abs(u[3])
    assert np.max(np.abs(sp.integral(sp.conv(u)))) < 1e-12
    assert np.max(np.abs(sp.integral(sp.lap(u)))) < 1e-11
    const = np.ones(sp.shape) * np.array([1.0, 0.3, -0.2, 2.5][:sp.ncomp])[:, None, None, None, None]
    assert np.max(np.abs(sp.conv(const))) < 1e-12
    assert np.max(np.abs(sp.lap(const))) < 1e-10
