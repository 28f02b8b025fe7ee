"""Seeded synthetic workloads: problem set-ups and initial data.

This module holds no arithmetic of the time-integration method or of the
spatial discretization.  It describes the workloads (PDE, domain, element
grids, polynomial degrees, collocation node sets, time step rule) and
evaluates closed-form initial data at node coordinates that the caller
supplies.  The same functions feed both the CUDA library and the CPU
oracle, so both see bit-identical inputs.

Random numbers come from numpy's PCG64 generator with seed
2504185260 + workload id.
"""
import math

import numpy as np

SEED_BASE = 2504185260


def rng_for(workload_id, extra=0):
    return np.random.default_rng(SEED_BASE + int(workload_id) + 1000 * int(extra))


# ---------------------------------------------------------------------------
# Workload descriptions (the five synthetic set-ups)
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 1D linear convection-diffusion, exact damped/shifted Fourier modes
    "convdiff1d": dict(
        id=1, pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=0.01,
        lo=(0.0, 0.0), hi=(2 * math.pi, 0.0),
        levels=[dict(nel=(16, 1), P=2, M=3), dict(nel=(16, 1), P=4, M=5)],
        nodes="lobatto", dt=0.05, nsteps=40, ncycles=4, start="cascade"),
    # 2D viscous Burgers, 2 components, 32x32 elements, P = 7
    "burgers2d": dict(
        id=2, pde="burgers", dim=2, ncomp=2, nu=5e-3,
        lo=(0.0, 0.0), hi=(1.0, 1.0),
        levels=[dict(nel=(32, 32), P=3, M=3), dict(nel=(32, 32), P=7, M=5)],
        nodes="radau_right", cfl=0.5, nsteps=100, ncycles=3, start="cascade",
        fourier_K=4, fourier_amp=0.05),
    # 2D Euler isentropic vortex, 64x64 elements, P = 7/5/3
    "euler_vortex": dict(
        id=3, pde="euler", dim=2, ncomp=4, gamma=1.4,
        lo=(-10.0, -10.0), hi=(10.0, 10.0),
        levels=[dict(nel=(64, 64), P=3, M=2), dict(nel=(64, 64), P=5, M=3),
                dict(nel=(64, 64), P=7, M=5)],
        nodes="lobatto", cfl=0.5, nsteps=200, ncycles=3, start="fmg1",
        vortex_beta=5.0, mach=0.5, angle_deg=45.0),
    # the same Euler vortex on 256x256 elements (4.2 M nodes x 4 variables): a
    # size whose level arrays do not fit in L2
    "euler256": dict(
        id=6, pde="euler", dim=2, ncomp=4, gamma=1.4,
        lo=(-10.0, -10.0), hi=(10.0, 10.0),
        levels=[dict(nel=(256, 256), P=3, M=2), dict(nel=(256, 256), P=5, M=3),
                dict(nel=(256, 256), P=7, M=5)],
        nodes="lobatto", cfl=0.5, nsteps=20, ncycles=3, start="fmg1",
        vortex_beta=5.0, mach=0.5, angle_deg=45.0),
    # 2D compressible Navier-Stokes doubly periodic shear layer, 128x128 elements, P = 5
    "ns_shear": dict(
        id=4, pde="ns", dim=2, ncomp=4, gamma=1.4, Re=2500.0, Pr=0.72, mach=0.3,
        lo=(0.0, 0.0), hi=(1.0, 1.0),
        levels=[dict(nel=(128, 128), P=3, M=3), dict(nel=(128, 128), P=5, M=5)],
        nodes="radau_right", cfl=0.5, nsteps=100, ncycles=3, start="cascade",
        shear_delta=1.0 / 80.0, perturb_amp=0.05),
    # the viscous Burgers moving front (Sec. 8, the spatially under-resolved case:
    # 10/20/40 elements of degree 8) as the x-momentum u_1 = w / 2 of the
    # two-component Burgers system on one element row (u_2 = 0, data constant
    # in y), with the artificial viscosity d_s = c_s = 0.5
    "burgers_front": dict(
        id=7, pde="burgers", dim=2, ncomp=2, nu=1e-2,
        lo=(-1.0, 0.0), hi=(1.0, 2.0),
        levels=[dict(nel=(10, 1), P=8, M=3), dict(nel=(20, 1), P=8, M=5), dict(nel=(40, 1), P=8, M=7)],
        nodes="radau_right", T=0.1, start="fmg1", av=dict(kappa=0.5, cs=0.5, comp=0),
        window=(-0.75, 0.75)),
    # Sod's shock tube (Sec. 8: 80 elements of degree 5/3 on [0, 1], M = 7/5, 32
    # steps to t = 0.2, Cascade start, d_s = 2, c_s = 0.4) mirrored to the
    # periodic [0, 2] (walls at x = 0 and 1 by symmetry) on one element row
    "sod": dict(
        id=8, pde="euler", dim=2, ncomp=4, gamma=1.4,
        lo=(0.0, 0.0), hi=(2.0, 2.0),
        levels=[dict(nel=(160, 1), P=3, M=5), dict(nel=(160, 1), P=5, M=7)],
        nodes="radau_right", T=0.2, nsteps=32, start="cascade", av=dict(kappa=2.0, cs=0.4, comp=0)),
    # 512 independent 2D convection-diffusion problems of mixed sizes and degrees
    "ensemble512": dict(
        id=5, pde="convdiff", dim=2, ncomp=1, ninst=512, nel_range=(8, 48), P_range=(3, 8),
        nu_range=(1e-4, 1e-2), fourier_K=6, fourier_amp=1.0, cfl=0.5,
        M=5, Mc=3, nodes="radau_right", nsteps=100, ncycles=3, start="cascade"),
}


# ---------------------------------------------------------------------------
# Closed-form initial data
# ---------------------------------------------------------------------------
def convdiff1d_exact(X, t, nu=0.01, a=1.0):
    """u = e^{-nu t} sin(x - a t) + 0.5 e^{-9 nu t} sin(3 (x - a t))."""
    return (np.exp(-nu * t) * np.sin(X - a * t)
            + 0.5 * np.exp(-9.0 * nu * t) * np.sin(3.0 * (X - a * t)))[None]


def fourier_modes(rng, K, ncomp):
    """All integer (kx, ky) != 0 with |k| <= K; per component a, b ~ U[-1, 1]."""
    modes = []
    for kx in range(-K, K + 1):
        for ky in range(-K, K + 1):
            if (kx, ky) == (0, 0) or kx * kx + ky * ky > K * K:
                continue
            a = rng.uniform(-1.0, 1.0, size=ncomp)
            b = rng.uniform(-1.0, 1.0, size=ncomp)
            modes.append((kx, ky, a, b))
    return modes


def eval_fourier(modes, X, Y, amp, ncomp):
    out = np.zeros((ncomp,) + X.shape)
    for kx, ky, a, b in modes:
        ph = 2.0 * math.pi * (kx * X + ky * Y)
        c, s = np.cos(ph), np.sin(ph)
        for q in range(ncomp):
            out[q] += amp * (a[q] * c + b[q] * s)
    return out


def burgers2d_initial(X, Y, seed_extra=0, K=4, amp=0.05):
    base = np.stack([np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y),
                     -np.cos(2 * math.pi * X) * np.sin(2 * math.pi * Y)])
    modes = fourier_modes(rng_for(2, seed_extra), K, 2)
    return base + eval_fourier(modes, X, Y, amp, 2)


def isentropic_vortex(X, Y, t=0.0, gamma=1.4, beta=5.0, mach=0.5, angle_deg=45.0,
                      lo=(-10.0, -10.0), hi=(10.0, 10.0)):
    """Conserved variables of the isentropic vortex translated by v_inf t on
    the periodic box (free stream rho = p = 1, |v_inf| = Mach * sqrt(gamma))."""
    vinf = mach * math.sqrt(gamma)
    ang = math.radians(angle_deg)
    vx0, vy0 = vinf * math.cos(ang), vinf * math.sin(ang)
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    # vortex centre at the origin at t = 0, moved by v_inf t, wrapped
    xc = (0.0 + vx0 * t - lo[0]) % Lx + lo[0]
    yc = (0.0 + vy0 * t - lo[1]) % Ly + lo[1]
    dx = (X - xc + Lx / 2) % Lx - Lx / 2
    dy = (Y - yc + Ly / 2) % Ly - Ly / 2
    r2 = dx * dx + dy * dy
    f = beta / (2 * math.pi) * np.exp(0.5 * (1.0 - r2))
    vx = vx0 - dy * f
    vy = vy0 + dx * f
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    return np.stack([rho, rho * vx, rho * vy, E])


def shear_layer(X, Y, gamma=1.4, mach=0.3, delta=1.0 / 80.0, amp=0.05, seed_extra=0):
    """Conserved variables of the doubly periodic shear layer on [0,1]^2:
    rho = 1, v_x = tanh((y - 1/4)/delta) for y <= 1/2 and tanh((3/4 - y)/delta)
    above, v_y = amp sin(2 pi (x + phi)) with a seeded phase phi in [0, 1),
    p = 1 / (gamma Mach^2)."""
    phi = float(rng_for(4, seed_extra).uniform(0.0, 1.0))
    vx = np.where(Y <= 0.5, np.tanh((Y - 0.25) / delta), np.tanh((0.75 - Y) / delta))
    vy = amp * np.sin(2.0 * math.pi * (X + phi))
    rho = np.ones_like(X)
    p = np.full_like(X, 1.0 / (gamma * mach * mach))
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    return np.stack([rho, rho * vx, rho * vy, E])


def max_wave_speed(pde, u, gamma=1.4, adv=(1.0, 0.0)):
    """Largest characteristic speed of the initial data (sets dt from CFL)."""
    if pde == "convdiff":
        return max(abs(adv[0]), abs(adv[1]))
    if pde == "burgers":
        return float(2.0 * np.max(np.abs(u)))
    if pde in ("euler", "ns"):
        rho = u[0]
        vx, vy = u[1] / rho, u[2] / rho
        p = (gamma - 1.0) * (u[3] - 0.5 * rho * (vx * vx + vy * vy))
        c = np.sqrt(gamma * p / rho)
        return float(max(np.max(np.abs(vx) + c), np.max(np.abs(vy) + c)))
    raise ValueError(pde)


_DELTA = {}


def cfl_delta(P):
    """delta of the CFL definition (Sec. 8): the largest eigenvalue magnitude
    of the convection problem u_t + u_x = 0 on the standard element [-1, 1]
    with a one-sided (inflow) Dirichlet condition, in the degree-P GLL
    collocation discretization -- the derivative matrix on the P+1 GLL
    nodes with the inflow node removed.  It grows like P^2 (about 0.09-0.15
    P^2 for P = 4..15)."""
    if P not in _DELTA:
        n = P + 1
        # GLL nodes: -1, 1 and the roots of P_P'
        inner = np.polynomial.legendre.Legendre.basis(P).deriv().roots().real if P > 1 else np.array([])
        x = np.concatenate([[-1.0], np.sort(inner), [1.0]])
        # derivative matrix of the Lagrange basis on x (barycentric weights)
        bw = np.array([1.0 / np.prod([x[j] - x[k] for k in range(n) if k != j]) for j in range(n)])
        D = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                if i != j:
                    D[i, j] = (bw[j] / bw[i]) / (x[i] - x[j])
            D[i, i] = -np.sum(D[i])
        _DELTA[P] = float(np.max(np.abs(np.linalg.eigvals(D[1:, 1:]))))
    return _DELTA[P]


def cfl_dt(cfl, h_elem, P, speed):
    """dt = CFL * dx / lam_max with dx = h_e / (2 delta), delta = cfl_delta(P)
    (the CFL definition of the numerical experiments, Sec. 8)."""
    return cfl * (h_elem / (2.0 * cfl_delta(P))) / speed


def burgers_front(X, t, nu=1e-2):
    """Exact moving front of w_t + (w^2/2)_x = nu w_xx, w = 1 - tanh((x + 0.5 - t) / (2 nu))
    (Sec. 8), as the state (u_1, u_2) = (w / 2, 0) of the two-component Burgers
    system, whose x-momentum equation u_t + (u^2)_x = nu u_xx it solves."""
    X = np.asarray(X, dtype=float)
    return np.stack([0.5 * (1.0 - np.tanh((X + 0.5 - t) / (2.0 * nu))), np.zeros_like(X)])


def _sod_star(gamma=1.4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Pressure and velocity between the two nonlinear waves of a Riemann
    problem of the Euler equations (Newton iteration on the pressure
    function of the exact solution, both waves as shocks or rarefactions)."""
    g = gamma
    (rl, ul, pl), (rr, ur, pr) = left, right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:                                   # shock
            A, B = 2.0 / ((g + 1.0) * rk), (g - 1.0) / (g + 1.0) * pk
            s = math.sqrt(A / (p + B))
            return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
        r = (p / pk) ** ((g - 1.0) / (2.0 * g))      # rarefaction
        return 2.0 * ck / (g - 1.0) * (r - 1.0), r / (rk * ck)

    p = 0.5 * (pl + pr)
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        dp = (f1 + f2 + ur - ul) / (d1 + d2)
        p = max(1e-12, p - dp)
        if abs(dp) < 1e-15 * p:
            break
    f1, _ = fk(p, rl, pl, cl)
    f2, _ = fk(p, rr, pr, cr)
    return p, 0.5 * (ul + ur) + 0.5 * (f2 - f1)


def sod_primitive(x, t, gamma=1.4, x0=0.5):
    """Exact density, velocity and pressure of Sod's problem (left state
    rho = p = 1, right rho = 0.125, p = 0.1, at rest) at x, time t > 0:
    left rarefaction, contact, right shock."""
    g = gamma
    rl, pl, rr, pr = 1.0, 1.0, 0.125, 0.1
    cl = math.sqrt(g * pl / rl)
    ps, us = _sod_star(gamma)
    rls = rl * (ps / pl) ** (1.0 / g)                                  # isentropic behind the fan
    cls = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    q = ps / pr
    rrs = rr * (q + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * q + 1.0)
    S = math.sqrt(g * pr / rr) * math.sqrt((g + 1.0) / (2.0 * g) * q + (g - 1.0) / (2.0 * g))
    xi = (np.asarray(x, dtype=float) - x0) / t
    rho = np.where(xi < -cl, rl, 0.0)
    u = np.zeros_like(xi)
    p = np.where(xi < -cl, pl, 0.0)
    fan = (xi >= -cl) & (xi < us - cls)
    uf = 2.0 / (g + 1.0) * (cl + xi)
    cf = 2.0 / (g + 1.0) * cl - (g - 1.0) / (g + 1.0) * xi
    rho = np.where(fan, rl * (np.maximum(cf, 0.0) / cl) ** (2.0 / (g - 1.0)), rho)
    u = np.where(fan, uf, u)
    p = np.where(fan, pl * (np.maximum(cf, 0.0) / cl) ** (2.0 * g / (g - 1.0)), p)
    left_star = (xi >= us - cls) & (xi < us)
    right_star = (xi >= us) & (xi < S)
    right = xi >= S
    rho = np.where(left_star, rls, np.where(right_star, rrs, np.where(right, rr, rho)))
    u = np.where(left_star | right_star, us, np.where(right, 0.0, u))
    p = np.where(left_star | right_star, ps, np.where(right, pr, p))
    return rho, u, p


def sod_state(X, t, gamma=1.4):
    """Conserved variables of the mirrored Sod problem on the periodic [0, 2]
    at the nodes X[ey, ex, j, i]: Sod's solution on [0, 1], its mirror image
    (velocity reversed) on [1, 2].  At t = 0 every element takes the state
    of its centre, so the discontinuities sit on the element faces at
    x = 0.5 and 1.5."""
    X = np.asarray(X, dtype=float)
    if t == 0.0:
        xc = np.broadcast_to(X.mean(axis=(-2, -1), keepdims=True), X.shape)
        left = (xc < 0.5) | (xc >= 1.5)
        rho = np.where(left, 1.0, 0.125)
        u = np.zeros_like(X)
        p = np.where(left, 1.0, 0.1)
    else:
        xm = np.where(X <= 1.0, X, 2.0 - X)
        rho, u, p = sod_primitive(xm, t, gamma)
        u = np.where(X <= 1.0, u, -u)
    return np.stack([rho, rho * u, np.zeros_like(X), p / (gamma - 1.0) + 0.5 * rho * u * u])


def initial_state(name, X, Y, seed_extra=0):
    w = WORKLOADS[name]
    if name == "convdiff1d":
        return convdiff1d_exact(X, 0.0, w["nu"], w["adv"][0])
    if name == "burgers2d":
        return burgers2d_initial(X, Y, seed_extra, w["fourier_K"], w["fourier_amp"])
    if name in ("euler_vortex", "euler256"):
        return isentropic_vortex(X, Y, 0.0, w["gamma"], w["vortex_beta"], w["mach"],
                                 w["angle_deg"], w["lo"], w["hi"])
    if name == "ns_shear":
        return shear_layer(X, Y, w["gamma"], w["mach"], w["shear_delta"], w["perturb_amp"], seed_extra)
    if name == "burgers_front":
        return burgers_front(X, 0.0, w["nu"])
    if name == "sod":
        return sod_state(X, 0.0, w["gamma"])
    raise ValueError(name)


def scaled(name, nel=None, P=None, levels=None):
    """A copy of a workload with a different element grid (all levels) and/or
    level list, for small parity cases."""
    import copy
    w = copy.deepcopy(WORKLOADS[name])
    if levels is not None:
        w["levels"] = levels
    if nel is not None:
        for lv in w["levels"]:
            lv["nel"] = tuple(nel)
    return w


def ensemble_instances(n=512, nel_range=(8, 48), P_range=(3, 8), nu_range=(1e-4, 1e-2), cfl=0.5,
                       seed_extra=0):
    """n instance descriptions of the ensemble workload: element grid n_e x n_e
    with n_e ~ U{nel_range}, degree P ~ U{P_range}, nu log-uniform in nu_range,
    velocity (cos t, sin t) with t ~ U[0, 2 pi), dt from the CFL number on the
    instance's own grid; plus the seed of its initial data."""
    rng = rng_for(5, seed_extra)
    out = []
    for k in range(n):
        ne = int(rng.integers(nel_range[0], nel_range[1] + 1))
        P = int(rng.integers(P_range[0], P_range[1] + 1))
        nu = float(10.0 ** rng.uniform(math.log10(nu_range[0]), math.log10(nu_range[1])))
        th = float(rng.uniform(0.0, 2.0 * math.pi))
        adv = (math.cos(th), math.sin(th))
        dt = cfl_dt(cfl, 1.0 / ne, P, max(abs(adv[0]), abs(adv[1])))
        out.append(dict(nel=(ne, ne), P=P, nu=nu, adv=adv, dt=dt, seed=1 + k + 10000 * int(seed_extra)))
    return out


def ensemble_modes(inst, K=6, amp=1.0):
    """Fourier modes |k| <= K of one instance, amplitude amp / sqrt(#modes)
    (normalised so that the data's RMS does not grow with K)."""
    modes = fourier_modes(rng_for(5, inst["seed"]), K, 1)
    return modes, amp / math.sqrt(len(modes))


def ensemble_exact(inst, X, Y, t, K=6, amp=1.0):
    """Exact solution of u_t + a . grad u = nu lap u on the periodic unit square
    for the instance's Fourier data: every mode is shifted by a t and damped
    by exp(-4 pi^2 nu |k|^2 t).  a cos(phi) + b sin(phi) is evaluated as
    Re((a - i b) e^{i phi}) with e^{i phi} = e^{i 2 pi kx x} e^{i 2 pi ky y}."""
    modes, A = ensemble_modes(inst, K, amp)
    ax, ay = inst["adv"]
    Xs = np.asarray(X, dtype=float) - ax * t
    Ys = np.asarray(Y, dtype=float) - ay * t
    ex = {k: np.exp(2j * math.pi * k * Xs) for k in range(-K, K + 1)}
    ey = {k: np.exp(2j * math.pi * k * Ys) for k in range(-K, K + 1)}
    acc = np.zeros(Xs.shape, dtype=complex)
    for kx, ky, a, b in modes:
        damp = math.exp(-4.0 * math.pi ** 2 * inst["nu"] * (kx * kx + ky * ky) * t)
        acc += (A * damp * complex(a[0], -b[0])) * (ex[kx] * ey[ky])
    return acc.real[None]


# Wave packet of the paper's 1D convection-diffusion studies (the coefficient
# table of the preliminary studies, Sec. 7, reused in Sec. 8): rows
# (kappa / pi, a, s) of u = sum_i a_i sin(kappa_i (x - s_i - v t)) exp(-kappa_i^2 nu t)
# on the periodic unit interval.
WAVE_PACKET = ((2, 1.00, 0.00), (6, 1.50, 0.05), (10, 1.80, 0.10), (14, 1.70, 0.15),
               (18, 1.50, 0.20), (24, 1.30, 0.30), (30, 1.15, 0.18))


def wave_packet(X, t, nu, v=1.0):
    """The exact wave-packet solution at nodes X (returned with a leading
    component axis)."""
    X = np.asarray(X, dtype=float)
    u = np.zeros(X.shape)
    for kp, a, s in WAVE_PACKET:
        k = kp * math.pi
        u += a * np.sin(k * (X - s - v * t)) * math.exp(-k * k * nu * t)
    return u[None]


def random_field(shape, seed, scale=1.0):
    """Seeded smooth-free random nodal data for operator-level parity tests."""
    return scale * np.random.default_rng(SEED_BASE + 77 + int(seed)).standard_normal(shape)
