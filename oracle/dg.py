"""DG-SEM spatial operators on periodic uniform meshes, FP64 (test infrastructure only).

The paper (Sec. 6) states the DG-SEM space (polynomials of degree P per
element, average and jump operators) and defers the flux details to its
companion paper.  The readings implemented here (listed in the design notes):

* nodal GLL collocation, diagonal GLL mass M = (h_x/2 w_i)(h_y/2 w_j);
* convective operator c(u) = -div F_c(u) in strong form with a local
  Lax-Friedrichs (Rusanov) flux F* = 1/2 (F(u-) + F(u+)) n - 1/2 lam (u+ - u-),
  lam = max(rho(A_n(u-)), rho(A_n(u+))) per face node;
* diffusion by symmetric interior penalty (SIPG) with GLL quadrature on
  volumes and faces, penalty tau = 2 (P+1)^2 / h_perp;  L = -M^{-1} A;
* the "diffusion-type" implicit operator of the SI integrators (Sec. 3.3,
  eq. H_SI(1)) is nu_tilde * L with the scalar
  nu_tilde = nu_d + (dt_m / 2) lam_max(u_b)^2 (exact for 1D convection-
  diffusion, a reading for 2D systems).

Array layout: u[c, ey, ex, j, i] with i (x-node) fastest; 1D meshes use
ney = 1 and nqy = 1.

Pins: SIPG symmetric, positive semi-definite, A 1 = 0 (dense assembly);
strong form equals an independently written weak form; spectral accuracy on
smooth data; exact translating-vortex time derivative for Euler; discrete
mass conservation.
"""
import numpy as np

from .tables import gll, diff_matrix


# --------------------------------------------------------------------------
# PDE flux definitions (Sec. 2)
# --------------------------------------------------------------------------
class ConvDiff:
    """u_t + a . grad u = nu lap u (scalar)."""

    def __init__(self, a, nu):
        self.a = tuple(float(x) for x in a)
        self.nu = float(nu)
        self.ncomp = 1
        self.nu_d = self.nu

    def flux_x(self, u):
        return self.a[0] * u

    def flux_y(self, u):
        return self.a[1] * u

    def rho_x(self, u):
        return np.full(u.shape[1:], abs(self.a[0]))

    def rho_y(self, u):
        return np.full(u.shape[1:], abs(self.a[1]))


class Burgers2:
    """Two-component viscous Burgers in conservative form,
    F^x = (u1^2, u1 u2), F^y = (u1 u2, u2^2); eigenvalues of A_n are u.n and
    2 u.n, so rho(A_n) = 2 |u.n|."""

    def __init__(self, nu):
        self.nu = float(nu)
        self.ncomp = 2
        self.nu_d = self.nu

    def flux_x(self, u):
        return np.stack([u[0] * u[0], u[0] * u[1]])

    def flux_y(self, u):
        return np.stack([u[0] * u[1], u[1] * u[1]])

    def rho_x(self, u):
        return 2.0 * np.abs(u[0])

    def rho_y(self, u):
        return 2.0 * np.abs(u[1])


class Euler2:
    """2D compressible Euler, u = (rho, rho v_x, rho v_y, rho e_t), perfect gas
    (Sec. 2.2 with eta = lambda = 0)."""

    def __init__(self, gamma):
        self.gamma = float(gamma)
        self.ncomp = 4
        self.nu_d = 0.0
        self.nu = 0.0

    def pressure(self, u):
        r, mx, my, E = u
        return (self.gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / r)

    def flux_x(self, u):
        r, mx, my, E = u
        p = self.pressure(u)
        vx = mx / r
        return np.stack([mx, mx * vx + p, my * vx, (E + p) * vx])

    def flux_y(self, u):
        r, mx, my, E = u
        p = self.pressure(u)
        vy = my / r
        return np.stack([my, mx * vy, my * vy + p, (E + p) * vy])

    def sound(self, u):
        return np.sqrt(self.gamma * self.pressure(u) / u[0])

    def rho_x(self, u):
        return np.abs(u[1] / u[0]) + self.sound(u)

    def rho_y(self, u):
        return np.abs(u[2] / u[0]) + self.sound(u)


class NavierStokes2(Euler2):
    """2D compressible Navier-Stokes (Sec. 2.2): the Euler fluxes plus the
    viscous flux of a Newtonian fluid with Stokes' hypothesis and Fourier heat
    conduction, in units with gas constant 1: temperature T = p / rho,
    viscosity mu = 1 / Re, conductivity kappa = mu gamma / ((gamma - 1) Pr).
    Viscous flux F_v^x = (0, tau_xx, tau_xy, v_x tau_xx + v_y tau_xy + kappa T_x)
    (and F_v^y alike) with tau = mu (grad v + grad v^T - 2/3 div v I).
    The viscous term is explicit (in f only); the implicit diffusion-type term
    of the SI integrators uses the scalar nu_d = max(4/3, gamma / Pr) mu / rho_ref
    (reading: rho_ref = the smallest density of the initial data)."""

    def __init__(self, gamma, Re, Pr, rho_ref=1.0):
        super().__init__(gamma)
        self.mu = 1.0 / float(Re)
        self.Pr = float(Pr)
        self.kappa = self.mu * self.gamma / ((self.gamma - 1.0) * self.Pr)
        self.nu_d = max(4.0 / 3.0, self.gamma / self.Pr) * self.mu / float(rho_ref)
        self.viscous = True

    def primitive(self, u):
        """(v_x, v_y, T) at every node."""
        r = u[0]
        return np.stack([u[1] / r, u[2] / r, self.pressure(u) / r])

    def viscous_flux(self, W, gx, gy):
        """F_v^x, F_v^y from the primitive values W and their gradients."""
        vx, vy = W[0], W[1]
        div = gx[0] + gy[1]
        txx = self.mu * (2.0 * gx[0] - (2.0 / 3.0) * div)
        tyy = self.mu * (2.0 * gy[1] - (2.0 / 3.0) * div)
        txy = self.mu * (gy[0] + gx[1])
        zero = np.zeros_like(vx)
        Fx = np.stack([zero, txx, txy, vx * txx + vy * txy + self.kappa * gx[2]])
        Fy = np.stack([zero, txy, tyy, vx * txy + vy * tyy + self.kappa * gy[2]])
        return Fx, Fy


# --------------------------------------------------------------------------
# DG-SEM level
# --------------------------------------------------------------------------
class DGSpace:
    """One spatial level: periodic uniform mesh of nel elements, degree P."""

    def __init__(self, dim, nel, P, lo, hi, pde, cg_rtol=1e-14, cg_maxit=10000):
        self.dim = dim
        self.P = P
        self.pde = pde
        self.ncomp = pde.ncomp
        self.nex = int(nel[0])
        self.ney = int(nel[1]) if dim == 2 else 1
        self.hx = (hi[0] - lo[0]) / self.nex
        self.hy = (hi[1] - lo[1]) / self.ney if dim == 2 else 1.0
        self.lo = tuple(lo)
        self.hi = tuple(hi)
        self.x, self.w = gll(P)
        self.D = diff_matrix(self.x)
        self.nqx = P + 1
        self.nqy = P + 1 if dim == 2 else 1
        self.shape = (self.ncomp, self.ney, self.nex, self.nqy, self.nqx)
        self.cg_rtol = cg_rtol
        self.cg_maxit = cg_maxit
        self.last_cg_iters = []
        wy = self.w if dim == 2 else np.ones(1)
        hy2 = self.hy / 2.0 if dim == 2 else 1.0
        self.mass = (hy2 * wy)[:, None] * ((self.hx / 2.0) * self.w)[None, :]
        self.diagA = self._diag_A()
        # artificial viscosity (oracle.av): None, or dict(kappa=d_s, cs=c_s, comp=sensor component)
        self.av = None

    # ---- geometry -------------------------------------------------------
    def coords(self):
        """Node coordinates X[ey, ex, j, i], Y[ey, ex, j, i]."""
        ex = np.arange(self.nex)
        X = self.lo[0] + (ex[:, None] + (self.x[None, :] + 1.0) / 2.0) * self.hx   # (nex, nqx)
        X = np.broadcast_to(X[None, :, None, :], (self.ney, self.nex, self.nqy, self.nqx))
        if self.dim == 1:
            return X.copy(), np.zeros_like(X)
        ey = np.arange(self.ney)
        Y = self.lo[1] + (ey[:, None] + (self.x[None, :] + 1.0) / 2.0) * self.hy   # (ney, nqy)
        Y = np.broadcast_to(Y[:, None, :, None], (self.ney, self.nex, self.nqy, self.nqx))
        return X.copy(), Y.copy()

    def zeros(self):
        return np.zeros(self.shape)

    # ---- convective operator -------------------------------------------
    def conv(self, u):
        """c(u) = -div F_c(u): strong-form DG-SEM with Rusanov face flux."""
        pde, D, w = self.pde, self.D, self.w
        hx = self.hx
        c = -(2.0 / hx) * np.einsum('ik,...k->...i', D, pde.flux_x(u))
        uL = u[..., -1]                               # right trace of element ex
        uR = np.roll(u[..., 0], -1, axis=2)           # left trace of element ex+1
        FL, FR = pde.flux_x(uL), pde.flux_x(uR)
        lam = np.maximum(pde.rho_x(uL), pde.rho_x(uR))
        Fs = 0.5 * (FL + FR) - 0.5 * lam * (uR - uL)  # numerical flux in +x
        c[..., -1] -= (2.0 / hx) / w[-1] * (Fs - FL)
        c[..., 0] += (2.0 / hx) / w[0] * (np.roll(Fs, 1, axis=2) - pde.flux_x(u[..., 0]))
        if self.dim == 2:
            hy = self.hy
            c -= (2.0 / hy) * np.einsum('jk,...kx->...jx', D, pde.flux_y(u))
            uB = u[..., -1, :]                        # top trace of element ey
            uT = np.roll(u[..., 0, :], -1, axis=1)    # bottom trace of element ey+1
            GB, GT = pde.flux_y(uB), pde.flux_y(uT)
            lam = np.maximum(pde.rho_y(uB), pde.rho_y(uT))
            Gs = 0.5 * (GB + GT) - 0.5 * lam * (uT - uB)
            c[..., -1, :] -= (2.0 / hy) / w[-1] * (Gs - GB)
            c[..., 0, :] += (2.0 / hy) / w[0] * (np.roll(Gs, 1, axis=1) - pde.flux_y(u[..., 0, :]))
        return c

    # ---- SIPG diffusion ---------------------------------------------------
    def penalty(self, h):
        return 2.0 * (self.P + 1) ** 2 / h

    def _sipg_line(self, v, h):
        """1D periodic SIPG stiffness along the last two axes (element, node)."""
        D, w = self.D, self.w
        K = D.T @ (w[:, None] * D)
        tau = self.penalty(h)
        out = (2.0 / h) * np.einsum('ik,...ek->...ei', K, v)
        dR = (2.0 / h) * (v @ D[-1])                  # u' at right end of each element
        dL = (2.0 / h) * (v @ D[0])                   # u' at left end
        jump = v[..., -1] - np.roll(v[..., 0], -1, axis=-1)   # [u] on interface e|e+1
        avg = 0.5 * (dR + np.roll(dL, -1, axis=-1))           # {u'} on interface e|e+1
        # element on the left of the interface
        out = out - (1.0 / h) * jump[..., None] * D[-1]
        out[..., -1] += -avg + tau * jump
        # element on the right of the interface
        out = out + np.roll(-(1.0 / h) * jump[..., None] * D[0], 1, axis=-2)
        out[..., 0] += np.roll(avg - tau * jump, 1, axis=-1)
        return out

    def A(self, u):
        """SIPG stiffness applied per component (a(u, .) as a nodal vector)."""
        ax = np.moveaxis(self._sipg_line(np.moveaxis(u, 3, 2), self.hx), 2, 3)
        if self.dim == 1:
            return ax
        out = ax * ((self.hy / 2.0) * self.w)[:, None]
        ay = self._sipg_line(u.transpose(0, 2, 4, 1, 3), self.hy).transpose(0, 3, 1, 4, 2)
        out = out + ay * ((self.hx / 2.0) * self.w)[None, :]
        return out

    def _diag_line(self, h):
        D, w = self.D, self.w
        K = D.T @ (w[:, None] * D)
        tau = self.penalty(h)
        d = (2.0 / h) * np.diag(K).copy()
        d[-1] += -2.0 * D[-1, -1] / h + tau
        d[0] += 2.0 * D[0, 0] / h + tau
        return d

    def _diag_A(self):
        dx = self._diag_line(self.hx)
        if self.dim == 1:
            return dx[None, :]
        dy = self._diag_line(self.hy)
        return ((self.hy / 2.0) * self.w)[:, None] * dx[None, :] + \
            dy[:, None] * ((self.hx / 2.0) * self.w)[None, :]

    def lap(self, u):
        """L u = -M^{-1} A u."""
        return -self.A(u) / self.mass

    def diff(self, u):
        """Diffusion term of f: nu L u, or the Navier-Stokes viscous term
        (zero for Euler), plus the artificial viscosity term when set."""
        if getattr(self.pde, "viscous", False):
            out = self.visc(u)
        elif self.pde.nu == 0.0:
            out = np.zeros_like(u)
        else:
            out = self.pde.nu * self.lap(u)
        if self.av is not None:
            from . import av
            out = out + av.av_term(self, u, av.viscosity(self, u, **self.av))
        return out

    @property
    def av_nu_lam(self):
        """c_s h / P: the artificial viscosity's share of nu_tilde per unit of
        lam_max (0 without artificial viscosity)."""
        if self.av is None:
            return 0.0
        from . import av
        return self.av["cs"] * av.h_min(self) / self.P

    # ---- viscous term (BR1) -------------------------------------------------
    def _lift_derivative(self, v, axis, h, sign):
        """Strong-form DG derivative of v along x (axis=-1) or y (axis=-2)
        with central face values {v} (Bassi-Rebay 1):
        (2/h) D v + (2/h)/w_P (v* - v) at the upper end - (2/h)/w_0 (v* - v)
        at the lower end, v* the average of the two traces; `sign` = +1
        (the same form serves the gradient and the divergence)."""
        D, w = self.D, self.w
        if axis == -1:
            d = (2.0 / h) * np.einsum('ik,...k->...i', D, v)
            up, lo = v[..., -1], v[..., 0]                           # [..., ey, ex, j]
            star = 0.5 * (up + np.roll(lo, -1, axis=-2))          # interface e | e+1 (x)
            d[..., -1] += sign * (2.0 / h) / w[-1] * (star - up)
            d[..., 0] -= sign * (2.0 / h) / w[0] * (np.roll(star, 1, axis=-2) - lo)
        else:
            d = (2.0 / h) * np.einsum('jk,...kx->...jx', D, v)
            up, lo = v[..., -1, :], v[..., 0, :]                     # [..., ey, ex, i]
            star = 0.5 * (up + np.roll(lo, -1, axis=-3))          # interface e | e+1 (y)
            d[..., -1, :] += sign * (2.0 / h) / w[-1] * (star - up)
            d[..., 0, :] -= sign * (2.0 / h) / w[0] * (np.roll(star, 1, axis=-3) - lo)
        return d

    def visc(self, u):
        """div F_v(u, grad u) by BR1: lifted gradients of the primitive
        variables with central traces, then the divergence of the viscous flux
        with central face fluxes (both in strong form)."""
        pde = self.pde
        W = pde.primitive(u)                                        # [3, ey, ex, j, i]
        gx = self._lift_derivative(W, -1, self.hx, 1.0)
        gy = self._lift_derivative(W, -2, self.hy, 1.0)
        Fx, Fy = pde.viscous_flux(W, gx, gy)
        return self._lift_derivative(Fx, -1, self.hx, 1.0) + self._lift_derivative(Fy, -2, self.hy, 1.0)

    @property
    def nu_d(self):
        return self.pde.nu_d

    def lam_max(self, u):
        """max over nodes of the convective spectral radius in x and y."""
        lm = np.max(self.pde.rho_x(u))
        if self.dim == 2:
            lm = max(lm, np.max(self.pde.rho_y(u)))
        return float(lm)

    # ---- implicit solve ---------------------------------------------------
    def solve(self, c, rhs, x0):
        """Solve (I - c L) x = rhs, i.e. (M + c A) x = M rhs, by Jacobi-PCG."""
        from .solver import pcg
        if c == 0.0:
            self.last_cg_iters.append(0)
            return rhs.copy()
        M = self.mass
        x, it = pcg(lambda v: M * v + c * self.A(v), M + c * self.diagA,
                    M * rhs, x0, self.cg_rtol, self.cg_maxit)
        self.last_cg_iters.append(it)
        return x

    # ---- diagnostics ------------------------------------------------------
    def l2(self, e):
        """Continuous L2 norm by GLL quadrature, summed over components."""
        return float(np.sqrt(np.sum(self.mass * e * e)))

    def integral(self, u):
        """Discrete mass sum_e sum_ij J w_i w_j u per component."""
        return np.sum(self.mass * u, axis=(1, 2, 3, 4))
