"""Pins of the oracle's artificial viscosity (oracle/av.py) and of the exact
reference solutions of the shock-capturing workloads (the Burgers moving
front and Sod's shock tube of Sec. 8).

The oracle's form of the Persson-Peraire viscosity is a reading (the paper
defers it to its companion); these tests pin each ingredient to something
outside the oracle: scipy's Legendre polynomials and Gauss quadrature,
closed-form modal energies, a manufactured solution of div(eps grad u) with
a viscosity jump at element faces, the algebraic properties of a
central-flux BR1 operator (conservation, symmetry, definiteness), and the
textbook star state of Sod's problem."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import av
from oracle.dg import DGSpace, ConvDiff, Burgers2, Euler2
from oracle.sdc import nutilde
from paper_2504_18526_gb300 import inputs


def _orthonormal(k, x):
    return math.sqrt((2 * k + 1) / 2.0) * eval_legendre(k, x)


def test_legendre_orthonormal_matches_scipy_and_is_orthonormal():
    x = np.linspace(-1, 1, 37)
    L = av.legendre_orthonormal(9, x)
    for k in range(10):
        assert np.allclose(L[k], _orthonormal(k, x), rtol=0, atol=1e-13)
    g, w = np.polynomial.legendre.leggauss(12)
    G = av.legendre_orthonormal(9, g)
    assert np.allclose((G * w) @ G.T, np.eye(10), atol=1e-13)


@pytest.mark.parametrize("P", [2, 5, 8])
def test_modal_coefficients_of_legendre_modes(P):
    """V^-1 maps the nodal values of L~_k to the k-th unit vector."""
    sp = DGSpace(1, (1,), P, (0.0,), (1.0,), ConvDiff((1.0, 0.0), 0.0))
    for k in range(P + 1):
        q = _orthonormal(k, sp.x)[None, None, None, :]
        c = av.modal_coefficients(sp, q)[0, 0, 0]
        e = np.zeros(P + 1)
        e[k] = 1.0
        assert np.allclose(c, e, atol=1e-12)


def test_sensor_closed_forms_1d():
    P = 6
    sp = DGSpace(1, (2,), P, (0.0,), (1.0,), ConvDiff((1.0, 0.0), 0.0))
    a, b = 0.3, 1.7
    q = np.stack([a * _orthonormal(P, sp.x) + b * _orthonormal(2, sp.x),
                  np.polyval([0.5, -1.0, 0.25, 2.0], sp.x)])[None, :, None, :]      # [ey, ex, j, i]
    S = av.sensor(sp, q)
    assert S[0, 0] == pytest.approx(a * a / (a * a + b * b), rel=1e-12)
    assert abs(S[0, 1]) < 1e-26                       # degree 3 < P: no energy in the top mode
    assert av.sensor(sp, np.zeros_like(q))[0, 0] == 0.0


def test_sensor_closed_form_2d_shell():
    """Tensor modes with max(k, l) = P form the top shell."""
    P = 4
    sp = DGSpace(2, (1, 1), P, (0.0, 0.0), (1.0, 1.0), Burgers2(0.0))
    x = sp.x
    a, b, c = 0.7, -1.1, 0.4
    q = (a * np.outer(_orthonormal(1, x), _orthonormal(P, x))          # y degree 1, x degree P
         + b * np.outer(_orthonormal(2, x), _orthonormal(3, x))
         + c * np.outer(_orthonormal(P, x), _orthonormal(0, x)))       # [j, i]
    S = av.sensor(sp, q[None, None])
    assert S[0, 0] == pytest.approx((a * a + c * c) / (a * a + b * b + c * c), rel=1e-12)


def test_ramp_end_values_and_midpoint():
    s0, k = -3.0, 0.5
    r = av.ramp(np.array([-10.0, s0 - k, s0 - 0.5 * k, s0, s0 + 0.5 * k, s0 + k, 10.0]), s0, k)
    assert r[0] == 0.0 and r[-1] == 1.0
    assert abs(r[1]) < 1e-16 and r[5] == pytest.approx(1.0, abs=1e-16)
    assert r[3] == pytest.approx(0.5, abs=1e-16)
    assert r[2] == pytest.approx(0.5 * (1 - math.sqrt(0.5)), rel=1e-14)
    assert r[4] == pytest.approx(0.5 * (1 + math.sqrt(0.5)), rel=1e-14)
    s = np.linspace(s0 - 2 * k, s0 + 2 * k, 401)
    assert np.all(np.diff(av.ramp(s, s0, k)) >= 0.0)


def test_viscosity_of_step_and_of_smooth_data():
    """A jump inside an element switches the viscosity fully on (eps0 = c_s h/P
    lam_e, lam_e = 2 max|u_1| for Burgers); smooth data leaves it off."""
    P, ne = 6, 8
    sp = DGSpace(2, (ne, 1), P, (0.0, 0.0), (1.0, 1.0), Burgers2(0.0))
    X, _ = sp.coords()
    u = np.zeros(sp.shape)
    u[0] = np.where(X < 0.3, 1.5, 0.25)                 # jump inside element 2 (0.25 .. 0.375)
    eps = av.viscosity(sp, u, kappa=0.5, cs=0.5, comp=0)
    h = min(sp.hx, sp.hy)
    assert eps[0, 2] == pytest.approx(0.5 * h / P * 2 * 1.5, rel=1e-14)
    assert np.all(np.delete(eps[0], 2) == 0.0)
    u[0] = 1.0 + 0.2 * np.sin(2 * np.pi * X)
    assert np.all(av.viscosity(sp, u, kappa=0.5, cs=0.5, comp=0) == 0.0)


def _jump_case(P, ne=4, e1=0.3, e2=0.05, slip=False):
    """div(eps grad u) for eps = e1 on [0, 1/2), e2 on [1/2, 1) and
    u = sin(2 pi x) / (2 pi eps(x)): eps u_x = cos(2 pi x) is smooth, so the
    exact result is -2 pi sin(2 pi x) although u_x jumps at x = 1/2."""
    sp = DGSpace(1, (ne,), P, (0.0,), (1.0,), ConvDiff((1.0, 0.0), 0.0))
    X, _ = sp.coords()
    xc = X.mean(axis=(-2, -1))                          # element centres [ey, ex]
    eps = np.where(xc < 0.5, e1, e2)
    epsn = np.broadcast_to(eps[:, :, None, None], X.shape)
    u = (np.sin(2 * np.pi * X) / (2 * np.pi * epsn))[None]
    if slip:                                            # planted: the neighbour's trace scaled by the own viscosity
        g = sp._lift_derivative(u, -1, sp.hx, 1.0)
        fl = eps[None, :, :, None, None] * g
        d = (2.0 / sp.hx) * np.einsum('ik,...k->...i', sp.D, fl)
        up, lo = fl[..., -1], fl[..., 0]
        nb_r = eps[None, :, :, None] * np.roll(g[..., 0], -1, axis=-2)
        nb_l = eps[None, :, :, None] * np.roll(g[..., -1], 1, axis=-2)
        d[..., -1] += (2.0 / sp.hx) / sp.w[-1] * (0.5 * (up + nb_r) - up)
        d[..., 0] -= (2.0 / sp.hx) / sp.w[0] * (0.5 * (nb_l + lo) - lo)
        out = d
    else:
        out = av.av_term(sp, u, eps)
    return np.max(np.abs(out[0] + 2 * np.pi * np.sin(2 * np.pi * X)))


def test_av_term_manufactured_viscosity_jump():
    e8, e12 = _jump_case(8), _jump_case(12)
    assert e12 < 1e-6
    assert e12 < e8 / 100.0
    assert _jump_case(12, slip=True) > 1.0              # a wrong face value is caught


@pytest.mark.parametrize("dim", [1, 2])
def test_av_term_conservative_symmetric_semidefinite(dim):
    rng = np.random.default_rng(11)
    P = 3
    if dim == 1:
        sp = DGSpace(1, (5,), P, (0.0,), (1.0,), ConvDiff((1.0, 0.0), 0.0))
    else:
        sp = DGSpace(2, (3, 2), P, (0.0, 0.0), (1.5, 1.0), ConvDiff((1.0, 0.5), 0.0))
    eps = rng.uniform(0.0, 2.0, (sp.ney, sp.nex))
    n = int(np.prod(sp.shape))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = (sp.mass * av.av_term(sp, e.reshape(sp.shape), eps)).ravel()
    assert np.allclose(A, A.T, atol=1e-11 * np.abs(A).max())
    assert np.max(np.linalg.eigvalsh(0.5 * (A + A.T))) < 1e-10 * np.abs(A).max()
    assert np.allclose(A.sum(axis=0), 0.0, atol=1e-11 * np.abs(A).max())      # conservation
    assert np.allclose(A @ np.ones(n), 0.0, atol=1e-11 * np.abs(A).max())     # constants in the kernel


def test_av_term_constant_viscosity_is_a_laplacian_2d():
    for P, tol in ((6, 1e-2), (10, 1e-6)):
        sp = DGSpace(2, (3, 3), P, (0.0, 0.0), (1.0, 1.0), ConvDiff((1.0, 0.0), 0.0))
        X, Y = sp.coords()
        u = (np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
        out = av.av_term(sp, u, np.full((3, 3), 0.7))
        assert np.max(np.abs(out + 0.7 * 8 * np.pi ** 2 * u)) < tol * 0.7 * 8 * np.pi ** 2


def test_nutilde_bounds_every_viscosity():
    """c_s h/P lam_max(u) >= eps_e for every element (the implicit coefficient covers it)."""
    rng = np.random.default_rng(5)
    sp = DGSpace(2, (6, 1), 5, (0.0, 0.0), (2.0, 2.0), Euler2(1.4))
    sp.av = dict(kappa=2.0, cs=0.4, comp=0)
    X, Y = sp.coords()
    u = inputs.sod_state(X, 0.0)
    u[0] *= 1.0 + 0.05 * rng.random(X.shape)
    eps = av.viscosity(sp, u, **sp.av)
    assert eps.max() > 0.0
    assert np.all(eps <= sp.av_nu_lam * sp.lam_max(u) * (1 + 1e-14))
    lam = sp.lam_max(u)
    assert nutilde(sp, u, 0.01) == pytest.approx(sp.nu_d + sp.av_nu_lam * lam + 0.005 * lam * lam, rel=1e-15)
    sp.av = None
    assert sp.av_nu_lam == 0.0


def test_sod_star_state_matches_the_textbook():
    """Star region of Sod's problem (Toro, Riemann Solvers and Numerical
    Methods for Fluid Dynamics, Sec. 4.3.3, test 1): p* = 0.30313,
    u* = 0.92745, rho*_L = 0.42632, rho*_R = 0.26557."""
    x = np.array([0.5 + 0.2 * 0.5, 0.5 + 0.2 * 1.2])       # left and right of the contact (u* t ~ 0.185)
    rho, u, p = inputs.sod_primitive(x, 0.2)
    assert p[0] == pytest.approx(0.30313, abs=1e-5) and p[1] == pytest.approx(0.30313, abs=1e-5)
    assert u[0] == pytest.approx(0.92745, abs=1e-5)
    assert rho[0] == pytest.approx(0.42632, abs=1e-5)
    assert rho[1] == pytest.approx(0.26557, abs=1e-5)


def test_sod_rankine_hugoniot_and_isentropic_fan():
    g = 1.4
    x = np.linspace(0.0, 1.0, 20001)
    rho, u, p = inputs.sod_primitive(x, 0.2)
    k = np.argmax(np.abs(np.diff(rho)) * (x[1:] > 0.75))     # the shock
    r1, u1, p1 = rho[k + 1], u[k + 1], p[k + 1]
    r2, u2, p2 = rho[k], u[k], p[k]
    S = (r2 * u2 - r1 * u1) / (r2 - r1)                      # shock speed from mass conservation
    mom = (r2 * u2 * (u2 - S) + p2) - (r1 * u1 * (u1 - S) + p1)
    E1 = p1 / (g - 1) + 0.5 * r1 * u1 * u1
    E2 = p2 / (g - 1) + 0.5 * r2 * u2 * u2
    en = (E2 * (u2 - S) + p2 * u2) - (E1 * (u1 - S) + p1 * u1)
    assert abs(mom) < 1e-10 and abs(en) < 1e-10
    fan = (x > 0.5 - 0.2 * math.sqrt(g)) & (x < 0.45)
    ent = p[fan] / rho[fan] ** g
    assert np.allclose(ent, 1.0, rtol=1e-12)
    assert np.all(np.diff(u[fan]) > 0)                        # accelerates through the fan


def test_mirrored_sod_state_is_symmetric():
    sp = DGSpace(2, (40, 1), 3, (0.0, 0.0), (2.0, 2.0), Euler2(1.4))
    X, _ = sp.coords()
    for t in (0.0, 0.13):
        s = inputs.sod_state(X, t)
        flip = s[:, :, ::-1, :, ::-1]                        # x -> 2 - x (elements and nodes reversed)
        assert np.allclose(s[0], flip[0]) and np.allclose(s[3], flip[3])
        assert np.allclose(s[1], -flip[1])
    s0 = inputs.sod_state(X, 0.0)
    assert s0[0, 0, 9].min() == 1.0 and s0[0, 0, 10].max() == 0.125       # jump on the face x = 0.5 (h = 0.05)


def test_burgers_front_solves_the_momentum_equation():
    """u_t + (u^2)_x = nu u_xx by central differences of the closed form."""
    nu, t, h = 1e-2, 0.05, 1e-4
    x = np.linspace(-0.8, 0.2, 41)
    u = lambda x, t: inputs.burgers_front(x, t, nu)[0]
    ut = (u(x, t + h) - u(x, t - h)) / (2 * h)
    fx = (u(x + h, t) ** 2 - u(x - h, t) ** 2) / (2 * h)
    uxx = (u(x + h, t) - 2 * u(x, t) + u(x - h, t)) / h ** 2
    assert np.max(np.abs(ut + fx - nu * uxx)) < 1e-3 * np.max(np.abs(ut))
    assert u(np.array([-1.0]), 0.0)[0] == pytest.approx(1.0) and u(np.array([1.0]), 0.0)[0] == pytest.approx(0.0)


def test_mlsdc_with_viscosity_converges_to_its_collocation_solution():
    """The viscosity is part of f: V-cycles of the front set-up (2:1
    h-coarsening, FMG_1 start, viscosity switched on by the steep front) drive
    the fine collocation residual F^nn(U) = U_m - U_{m-1} - dt S f(U), f with
    the viscosity term, towards zero (slowly: the scalar nu_tilde carries the
    viscosity's largest value into the smooth elements too); without the term
    in the sweeps' f (a planted slip) the iteration settles at a residual of
    the size of the term."""
    from oracle.sdc import Fnn
    from tests.helpers import oracle_ml
    w = inputs.scaled("burgers_front", levels=[dict(nel=(4, 1), P=4, M=3), dict(nel=(8, 1), P=4, M=3)])
    ml = oracle_ml(w, rtol=1e-14)
    fine = ml.levels[-1]
    X, _ = fine.space.coords()
    u0 = inputs.burgers_front(X, 0.0, w["nu"])
    assert av.viscosity(fine.space, u0, **w["av"]).max() > 0.0
    dt = 0.002
    res = []
    for nc in (4, 24):
        _, Us = ml.step(u0, dt, nc, start="fmg1", return_levels=True)
        res.append(np.max(np.abs(Fnn(fine, u0, Us[-1], dt))))
    assert res[1] < 1e-7 and res[1] < res[0] / 1000.0
    for lv in ml.levels:                                   # planted: f without the viscosity in the sweeps
        lv.space.av = None
    _, Us2 = ml.step(u0, dt, 24, start="fmg1", return_levels=True)
    for lv in ml.levels:
        lv.space.av = dict(w["av"])
    assert np.max(np.abs(Fnn(fine, u0, Us2[-1], dt))) > 1e-3
