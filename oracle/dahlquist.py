"""The scalar Fourier-mode (Dahlquist) problem of Sec. 5, run through the same
``sdc``/``mlsdc`` code as the DG problems (test infrastructure only).

For u = u_hat(t) e^{ikx} of u_t = -v u_x + nu u_xx with k = 1 the operators
reduce to c(u) = i lam_i u, L u = -u, nu_d = nu = -lam_r, lam_max = |lam_i|,
so that nu_tilde L = lam_r - dt_m lam_i^2 / 2 and the SI(1) substep factor is
(1 + i zeta_i) / (1 - zeta_r + zeta_i^2 / 2) with zeta = dt_m lam.
The stability function is R(z) = u^{n+1} / u^n for one step with dt = 1 and
u(0) = 1 (Sec. 5.1).
"""
import numpy as np

from .sdc import Level
from .mlsdc import MLSDC


class DahlquistSpace:
    def __init__(self, lam):
        self.lam = complex(lam)
        self.nu_d = -self.lam.real
        self.ncomp = 1

    def conv(self, u):
        return 1j * self.lam.imag * u

    def lap(self, u):
        return -u

    def diff(self, u):
        return self.lam.real * u

    def lam_max(self, u):
        return abs(self.lam.imag)

    def solve(self, c, rhs, x0):
        return rhs / (1.0 + c)


def stability(z, Ms, node_kind='radau_right', stages=2, ncycles=1, start='predictor',
              post_sweep=True, Nc=2, fmg_cycles=1):
    """R(z) of one SI-MLSDC step (levels with node counts Ms, coarse first)."""
    sp = DahlquistSpace(z)
    levels = [Level(sp, node_kind, M) for M in Ms]
    ml = MLSDC(levels, stages=stages, Nc=Nc, fmg_cycles=fmg_cycles)
    u1 = ml.step(np.complex128(1.0), 1.0, ncycles, start=start, post_sweep=post_sweep)
    return complex(u1)
