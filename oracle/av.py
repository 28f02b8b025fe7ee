"""Persson-Peraire artificial viscosity, FP64 (test infrastructure only).

The paper supplements the diffusion matrix of its DG right-hand side with the
artificial viscosity of Persson and Peraire to capture fronts and shocks
(Sec. 6, "Spatial discretization"; used for the Burgers moving front and the
Sod shock tube of Sec. 8 with the parameters d_s, c_s) and defers its form to
the companion paper.  The readings implemented here:

* sensor variable q: one component of the state (u_1 for Burgers, the
  density for Euler);
* modal decay per element: the element's GLL interpolant of q expanded in
  orthonormal Legendre polynomials (tensor products in 2D),
  S_e = (energy of the modes of the highest degree P, max(k, l) = P) /
  (energy of all modes), s_e = log10 S_e; S_e = 0 (q = 0 on the element)
  gives no viscosity;
* eps_e = eps0_e * ramp(s_e): 0 for s_e < s0 - kappa, eps0_e for
  s_e > s0 + kappa, eps0_e (1 + sin(pi (s_e - s0) / (2 kappa))) / 2 between;
  s0 = log10(1 / P^4), kappa = d_s, eps0_e = c_s h / P lam_e with h the
  smaller element side and lam_e the largest convective spectral radius over
  the element's nodes;
* the viscosity follows the state at which f is evaluated (every node and
  iterate), so it is part of f like the physical diffusion;
* the term div(eps grad u) acts on every component and is discretised by
  BR1: derivatives lifted with central face values, scaled by the element's
  eps, then the divergence with central face values (the form of the
  Navier-Stokes viscous term here);
* the implicit diffusion-type coefficient of the SI integrators covers it:
  nu_tilde = nu_d + c_s h / P lam_max + dt_m / 2 lam_max^2 (c_s h / P lam_max
  bounds every eps_e).

Pins (tests/test_oracle_av.py): modal energies of Legendre modes (against
scipy's Legendre polynomials), the ramp's end values and midpoint, a
manufactured solution with a viscosity jump at element faces, conservation,
symmetry and definiteness of the discrete operator, reduction to a constant
viscosity times the BR1 Laplacian.
"""
import math

import numpy as np

from .tables import gll


def legendre_orthonormal(n, x):
    """Orthonormal Legendre polynomials sqrt((2k+1)/2) P_k(x), k = 0..n, at x
    (Bonnet's three-term recurrence); shape (n + 1,) + x.shape."""
    x = np.asarray(x, dtype=float)
    L = np.zeros((n + 1,) + x.shape)
    L[0] = 1.0
    if n >= 1:
        L[1] = x
    for k in range(1, n):
        L[k + 1] = ((2 * k + 1) * x * L[k] - k * L[k - 1]) / (k + 1)
    return L * np.sqrt((2.0 * np.arange(n + 1) + 1.0) / 2.0).reshape((n + 1,) + (1,) * x.ndim)


def nodal_to_modal(P):
    """V^-1 with V[i, k] = L~_k(x_i) at the GLL nodes x_i: modal coefficients
    of the interpolant from nodal values."""
    x, _ = gll(P)
    V = legendre_orthonormal(P, x).T
    return np.linalg.inv(V)


def modal_coefficients(space, q):
    """Legendre coefficients c[..., l, k] (l: y degree, k: x degree) of q[..., j, i]."""
    Vi = nodal_to_modal(space.P)
    c = np.einsum('ki,...ji->...jk', Vi, q)
    if space.dim == 2:
        c = np.einsum('lj,...jk->...lk', Vi, c)
    return c


def sensor(space, q):
    """S_e = highest-degree modal energy / total modal energy per element
    (q[ey, ex, j, i] -> S[ey, ex]); 0 where q vanishes on the element."""
    c = modal_coefficients(space, q)
    e = c * c
    tot = e.sum(axis=(-2, -1))
    P = space.P
    if space.dim == 2:
        hi = e[..., P, :].sum(axis=-1) + e[..., :P, P].sum(axis=-1)
    else:
        hi = e[..., 0, P]
    return np.where(tot > 0.0, hi / np.where(tot > 0.0, tot, 1.0), 0.0)


def ramp(s, s0, kappa):
    """0 below s0 - kappa, 1 above s0 + kappa, (1 + sin(pi (s - s0) / (2 kappa))) / 2 between."""
    s = np.asarray(s, dtype=float)
    mid = 0.5 * (1.0 + np.sin(np.pi * np.clip(s - s0, -kappa, kappa) / (2.0 * kappa)))
    return np.where(s < s0 - kappa, 0.0, np.where(s > s0 + kappa, 1.0, mid))


def h_min(space):
    return space.hx if space.dim == 1 else min(space.hx, space.hy)


def element_lambda(space, u):
    """Largest convective spectral radius over each element's nodes, [ey, ex]."""
    r = space.pde.rho_x(u)
    if space.dim == 2:
        r = np.maximum(r, space.pde.rho_y(u))
    return r.max(axis=(-2, -1))


def viscosity(space, u, kappa, cs, comp=0):
    """eps_e per element [ey, ex] from the state u[c, ey, ex, j, i]."""
    P = space.P
    S = sensor(space, u[comp])
    with np.errstate(divide="ignore"):
        s = np.where(S > 0.0, np.log10(np.where(S > 0.0, S, 1.0)), -np.inf)
    s0 = math.log10(1.0 / P ** 4)
    eps0 = cs * h_min(space) / P * element_lambda(space, u)
    return eps0 * ramp(s, s0, kappa)


def av_term(space, u, eps):
    """div(eps grad u) per component by BR1 with the element-wise eps[ey, ex]."""
    e = eps[None, :, :, None, None]
    gx = space._lift_derivative(u, -1, space.hx, 1.0)
    out = space._lift_derivative(e * gx, -1, space.hx, 1.0)
    if space.dim == 2:
        gy = space._lift_derivative(u, -2, space.hy, 1.0)
        out = out + space._lift_derivative(e * gy, -2, space.hy, 1.0)
    return out
