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


# ---- Navier-Stokes viscous term (BR1) -----------------------------------------
def _ns_manufactured(g=1.4, Re=50.0, Pr=0.72):
    """A smooth periodic state and its viscous divergence, differentiated
    symbolically from the Newtonian stress and Fourier heat flux (T = p/rho)."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    rho = 1 + sp.Rational(1, 5) * sp.sin(2 * sp.pi * x) * sp.cos(2 * sp.pi * y)
    vx = sp.Rational(1, 2) * sp.sin(2 * sp.pi * y) + sp.Rational(1, 10) * sp.cos(2 * sp.pi * x)
    vy = sp.Rational(3, 10) * sp.cos(2 * sp.pi * (x + y))
    p = 2 + sp.Rational(1, 4) * sp.sin(2 * sp.pi * (x - y))
    T = p / rho
    mu = 1 / sp.Float(Re)
    kap = mu * g / ((g - 1) * Pr)
    div = sp.diff(vx, x) + sp.diff(vy, y)
    txx = mu * (2 * sp.diff(vx, x) - sp.Rational(2, 3) * div)
    tyy = mu * (2 * sp.diff(vy, y) - sp.Rational(2, 3) * div)
    txy = mu * (sp.diff(vx, y) + sp.diff(vy, x))
    Fx = [0, txx, txy, vx * txx + vy * txy + kap * sp.diff(T, x)]
    Fy = [0, txy, tyy, vx * txy + vy * tyy + kap * sp.diff(T, y)]
    exact = [sp.lambdify((x, y), sp.diff(Fx[k], x) + sp.diff(Fy[k], y), "numpy") for k in range(4)]
    cons = [sp.lambdify((x, y), e, "numpy")
            for e in (rho, rho * vx, rho * vy, p / (g - 1) + rho * (vx ** 2 + vy ** 2) / 2)]
    return exact, cons


def _ns_error(P, ne, exact, cons):
    from oracle.dg import NavierStokes2
    S = DGSpace(2, (ne, ne), P, (0.0, 0.0), (1.0, 1.0), NavierStokes2(1.4, 50.0, 0.72))
    X, Y = S.coords()
    u = np.stack([np.broadcast_to(c(X, Y), X.shape) for c in cons])
    v = S.visc(u)
    ex = np.stack([np.broadcast_to(np.asarray(e(X, Y), dtype=float), X.shape) for e in exact])
    return np.max(np.abs(v - ex)) / np.max(np.abs(ex)), S.integral(v), np.max(np.abs(v))


def test_ns_viscous_term_converges_to_symbolic_divergence():
    """BR1 viscous divergence against the symbolic div F_v of a manufactured
    state: converges under h- and p-refinement, 2e-6 at P = 8 on 8 x 8."""
    exact, cons = _ns_manufactured()
    e1, _, _ = _ns_error(6, 4, exact, cons)
    e2, _, _ = _ns_error(6, 8, exact, cons)
    e3, tot, scale = _ns_error(8, 8, exact, cons)
    assert e2 < 0.2 * e1 and e3 < 0.05 * e2 and e3 < 1e-5
    # central face fluxes telescope: every component integrates to zero
    assert np.all(np.abs(tot) <= 1e-14 * scale)


def test_ns_viscous_term_pure_shear():
    """rho = 1, v = (A sin 2 pi y, 0), p constant: momentum rate
    -mu A (2 pi)^2 sin 2 pi y, energy rate 4 pi^2 mu A^2 cos 4 pi y, nothing in
    y-momentum or mass."""
    from oracle.dg import NavierStokes2
    g, Re, A, p0 = 1.4, 100.0, 0.7, 3.0
    S = DGSpace(2, (6, 6), 8, (0.0, 0.0), (1.0, 1.0), NavierStokes2(g, Re, 0.72))
    X, Y = S.coords()
    vx = A * np.sin(2 * np.pi * Y)
    u = np.stack([np.ones_like(X), vx, np.zeros_like(X), p0 / (g - 1) + 0.5 * vx * vx])
    v = S.visc(u)
    mu = 1.0 / Re
    assert np.max(np.abs(v[0])) == 0.0
    assert np.max(np.abs(v[2])) < 1e-11
    assert np.max(np.abs(v[1] + mu * A * (2 * np.pi) ** 2 * np.sin(2 * np.pi * Y))) < 1e-6
    assert np.max(np.abs(v[3] - 4 * np.pi ** 2 * mu * A * A * np.cos(4 * np.pi * Y))) < 1e-5
