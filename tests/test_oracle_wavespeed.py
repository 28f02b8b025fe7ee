"""Pins for the oracle's Rusanov (local Lax-Friedrichs) wave speeds (CPU only).

The convective face flux of Sec. 6 uses lam = max(rho(A_n(u-)), rho(A_n(u+)))
with rho the spectral radius of the flux Jacobian A_n = d(F . n)/du.  The
oracle writes rho in closed form per PDE (rho_x, rho_y) and takes lam_max (the
largest one over the mesh, which feeds nu_tilde) from them.  Here they are
checked against what linear algebra fixes, independently of those formulas:

* the spectral radius of a central-difference Jacobian of the oracle's own
  flux functions (numpy eigenvalues), at random admissible states;
* the textbook eigenvalues of each system (Burgers u.n and 2 u.n; Euler
  v_n - c, v_n, v_n, v_n + c);
* a hand-computed Rusanov flux across a jump between two constant states,
  which must appear, lifted, in the end nodes of the strong-form operator;
* planted slips (|u.n| for Burgers, no sound speed for Euler, |v| for |v_n|)
  make the checks fail.
"""
import numpy as np
import pytest

from oracle.dg import Burgers2, ConvDiff, DGSpace, Euler2, NavierStokes2


def _states(pde, rng, n):
    """n random admissible states as an array [ncomp, n]."""
    if isinstance(pde, Euler2):
        rho = 0.3 + 2.0 * rng.random(n)
        vx, vy = rng.standard_normal(n), rng.standard_normal(n)
        p = 0.2 + 3.0 * rng.random(n)
        E = p / (pde.gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
        return np.stack([rho, rho * vx, rho * vy, E])
    return rng.standard_normal((pde.ncomp, n))


def _jacobian_radius(flux, u):
    """max |eig(dF/du)| at every column of u, by central differences."""
    nc, n = u.shape
    out = np.empty(n)
    for k in range(n):
        J = np.empty((nc, nc))
        for c in range(nc):
            h = 1e-6 * max(1.0, abs(u[c, k]))
            up, um = u[:, k:k + 1].copy(), u[:, k:k + 1].copy()
            up[c] += h
            um[c] -= h
            J[:, c] = (flux(up)[:, 0] - flux(um)[:, 0]) / (2.0 * h)
        out[k] = np.max(np.abs(np.linalg.eigvals(J)))
    return out


def _radius_deviation(pde, rng, n=40):
    """Largest relative gap between the oracle's rho_x/rho_y and the
    spectral radius of the finite-difference flux Jacobian."""
    u = _states(pde, rng, n)
    worst = 0.0
    for flux, rho in ((pde.flux_x, pde.rho_x), (pde.flux_y, pde.rho_y)):
        fd = _jacobian_radius(flux, u)
        r = np.broadcast_to(rho(u), fd.shape)
        worst = max(worst, float(np.max(np.abs(r - fd) / np.maximum(1.0, fd))))
    return worst


PDES = {
    "convdiff": lambda: ConvDiff((0.7, -1.3), 0.01),
    "burgers": lambda: Burgers2(0.0),
    "euler": lambda: Euler2(1.4),
    "ns": lambda: NavierStokes2(1.4, 2500.0, 0.72),
}


@pytest.mark.parametrize("name", list(PDES))
def test_rho_is_spectral_radius_of_flux_jacobian(name):
    assert _radius_deviation(PDES[name](), np.random.default_rng(11)) < 1e-7


def test_closed_form_eigenvalues():
    """Burgers: A_n has eigenvalues u.n and 2 u.n; Euler: v_n - c, v_n (twice),
    v_n + c with c = sqrt(gamma p / rho)."""
    rng = np.random.default_rng(5)
    b = Burgers2(0.0)
    u = _states(b, rng, 8)
    for k in range(8):
        for n, flux in (((1.0, 0.0), b.flux_x), ((0.0, 1.0), b.flux_y)):
            un = n[0] * u[0, k] + n[1] * u[1, k]
            J = np.empty((2, 2))
            for c in range(2):
                h = 1e-6
                up, um = u[:, k:k + 1].copy(), u[:, k:k + 1].copy()
                up[c] += h
                um[c] -= h
                J[:, c] = (flux(up)[:, 0] - flux(um)[:, 0]) / (2 * h)
            ev = np.sort(np.linalg.eigvals(J).real)
            assert np.allclose(ev, np.sort([un, 2.0 * un]), atol=1e-8)
    e = Euler2(1.4)
    u = _states(e, rng, 8)
    rho, vx, vy = u[0], u[1] / u[0], u[2] / u[0]
    p = 0.4 * (u[3] - 0.5 * rho * (vx * vx + vy * vy))
    c = np.sqrt(1.4 * p / rho)
    for k in range(8):
        for vn, flux in ((vx[k], e.flux_x), (vy[k], e.flux_y)):
            J = np.empty((4, 4))
            for q in range(4):
                h = 1e-6 * max(1.0, abs(u[q, k]))
                up, um = u[:, k:k + 1].copy(), u[:, k:k + 1].copy()
                up[q] += h
                um[q] -= h
                J[:, q] = (flux(up)[:, 0] - flux(um)[:, 0]) / (2 * h)
            ev = np.sort(np.linalg.eigvals(J).real)
            assert np.allclose(ev, np.sort([vn - c[k], vn, vn, vn + c[k]]), atol=1e-6)
        assert np.isclose(e.sound(u[:, k:k + 1])[0], c[k], rtol=1e-14)


@pytest.mark.parametrize("name", ["convdiff", "burgers", "euler"])
def test_lam_max_is_largest_radius_over_mesh(name):
    pde = PDES[name]()
    sp = DGSpace(2, (3, 2), 3, (0.0, 0.0), (1.0, 1.0), pde)
    rng = np.random.default_rng(2)
    n = int(np.prod(sp.shape[1:]))
    u = _states(pde, rng, n).reshape(sp.shape)
    flat = u.reshape(pde.ncomp, -1)
    want = max(np.max(_jacobian_radius(pde.flux_x, flat)), np.max(_jacobian_radius(pde.flux_y, flat)))
    assert abs(sp.lam_max(u) - want) < 1e-7 * max(1.0, want)


def _two_state_case(name, axis):
    """A 2D mesh of 2x2 elements whose state is constant per element, with a
    jump across the faces normal to `axis`; the left/bottom state has the
    larger wave speed on one face pair and the smaller on the other."""
    pde = PDES[name]()
    rng = np.random.default_rng(17 + axis)
    sA, sB = _states(pde, rng, 2).T
    sp = DGSpace(2, (2, 2), 3, (0.0, 0.0), (1.0, 2.0), pde)
    u = np.empty(sp.shape)
    for e in range(2):
        s = sA if e == 0 else sB
        if axis == 0:
            u[:, :, e] = s[:, None, None, None]
        else:
            u[:, e] = s[:, None, None, None]
    return pde, sp, u, sA, sB


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("name", ["convdiff", "burgers", "euler"])
def test_rusanov_face_flux_across_a_jump(name, axis):
    """Constant states per element: the volume term vanishes (D 1 = 0), so
    c(u) at the end nodes is the lifted difference of the hand-computed
    Rusanov flux F* = 1/2 (F(a) + F(b)) - 1/2 lam (b - a), lam the larger
    FD spectral radius of the two sides, and the trace flux."""
    pde, sp, u, sA, sB = _two_state_case(name, axis)
    flux = pde.flux_x if axis == 0 else pde.flux_y
    h = sp.hx if axis == 0 else sp.hy
    w = sp.w
    lift = (2.0 / h)

    def fstar(a, b):
        lam = max(_jacobian_radius(flux, a[:, None])[0], _jacobian_radius(flux, b[:, None])[0])
        return 0.5 * (flux(a[:, None])[:, 0] + flux(b[:, None])[:, 0]) - 0.5 * lam * (b - a)

    c = sp.conv(u)
    FA, FB = flux(sA[:, None])[:, 0], flux(sB[:, None])[:, 0]
    # face A|B (upper end of element 0) and the periodic face B|A (upper end of element 1)
    fAB, fBA = fstar(sA, sB), fstar(sB, sA)
    exp_A_hi = -lift / w[-1] * (fAB - FA)
    exp_B_lo = lift / w[0] * (fAB - FB)
    exp_B_hi = -lift / w[-1] * (fBA - FB)
    exp_A_lo = lift / w[0] * (fBA - FA)
    if axis == 0:
        got = (c[:, :, 0, :, -1], c[:, :, 1, :, 0], c[:, :, 1, :, -1], c[:, :, 0, :, 0])
    else:
        got = (c[:, 0, :, -1, :], c[:, 1, :, 0, :], c[:, 1, :, -1, :], c[:, 0, :, 0, :])
    scale = max(1.0, np.max(np.abs(c)))
    for g, e in zip(got, (exp_A_hi, exp_B_lo, exp_B_hi, exp_A_lo)):
        assert np.max(np.abs(g - e[:, None, None])) < 1e-7 * scale
    # interior nodes (away from the faces normal to axis) see no flux
    if axis == 0:
        assert np.max(np.abs(c[..., 1:-1])) < 1e-12 * scale
    else:
        assert np.max(np.abs(c[..., 1:-1, :])) < 1e-12 * scale


# ---- planted slips: each must be caught ----------------------------------
class _BurgersHalf(Burgers2):
    def rho_x(self, u):
        return np.abs(u[0])


class _EulerNoSound(Euler2):
    def rho_y(self, u):
        return np.abs(u[2] / u[0])


class _EulerSpeed(Euler2):
    def rho_x(self, u):
        return np.hypot(u[1], u[2]) / u[0] + self.sound(u)


@pytest.mark.parametrize("bad", [_BurgersHalf(0.0), _EulerNoSound(1.4), _EulerSpeed(1.4)])
def test_planted_wave_speed_slips_are_caught(bad):
    assert _radius_deviation(bad, np.random.default_rng(11)) > 1e-2


def test_planted_slip_changes_face_flux():
    """The face-flux check sees a wrong lam too: with Burgers' |u.n| in place
    of 2|u.n| the operator's end-node values move away from the hand flux."""
    good = DGSpace(2, (2, 2), 3, (0.0, 0.0), (1.0, 2.0), Burgers2(0.0))
    bad = DGSpace(2, (2, 2), 3, (0.0, 0.0), (1.0, 2.0), _BurgersHalf(0.0))
    _, _, u, _, _ = _two_state_case("burgers", 0)
    assert np.max(np.abs(good.conv(u) - bad.conv(u))) > 1e-3
