"""Multilevel SDC with FAS: transfers, V-cycle, Cascade/FMG starts, time step
(FP64, test infrastructure only).

* Transfers (Sec. 4.2, Sec. 6.2): space-time tensor products of the time
  transfers I_t, P_t, R_t = I_t^T and per-direction spatial transfers I_x,
  P_x (embedded interpolation, or the L2 projection) and R_x, for
  p-coarsening on the same elements and for 2:1 h-coarsening (two fine
  elements per coarse element and direction, tables.h_transfers).
* FAS right-hand side (Sec. 4.1, eq. ml-cm:incremental:fas-mg:rhs):
  g_l = F_l(P u_{l+1}) + R (g_{l+1} - F_{l+1}(u_{l+1})), g_L = 0.
* V-cycle: Algorithm 2.  Reading: after the solution restriction
  v_{l-1} = P u_l the coarse iterate is set to v_{l-1} (full approximation
  scheme), so that u_l += I(u_{l-1} - v_{l-1}) interpolates a correction.
* Starts: Algorithm 3 (Cascade), Algorithm 4 (FMG with C_fmg cycles per
  added level, default 1),
  predictor on all levels, constant spread of u_0 (Sec. 4.7).
* One step: start, C V-cycles, optional final fine post-sweep; the new
  value is u_{L,M} (t_M = t + dt for Radau-Right and Lobatto).
* Reading: the initial value of a coarse level is the spatial projection
  of the finer level's initial value (identical when only time coarsens).
"""
import numpy as np

from .sdc import corrector, corrector_0n, predictor, Fnn, F0n
from .tables import time_transfers, space_transfers, l2_projection, h_transfers


def _apply_space(mat, u, dim):
    """Apply a per-direction element matrix along x (and y) of u[..., j, i]."""
    out = np.einsum('ai,...i->...a', mat, u)
    if dim == 2:
        out = np.einsum('bj,...ja->...ba', mat, out)
    return out


def _apply_dir(mats, u, ax_e, ax_n, coarse_to_fine):
    """One direction of a transfer between element grids of ratio r =
    len(mats) (1: same elements, 2: 2:1 h-coarsening).  Coarse to fine:
    fine element e takes mats[e % r] applied to coarse element e // r.  Fine
    to coarse: coarse element e sums mats[c] applied to fine element r e + c."""
    r = len(mats)
    a = np.moveaxis(u, (ax_e, ax_n), (-2, -1))
    if coarse_to_fine:
        out = np.zeros(a.shape[:-2] + (a.shape[-2] * r, mats[0].shape[0]))
        for c in range(r):
            out[..., c::r, :] = np.einsum('ba,...ea->...eb', mats[c], a)
    else:
        out = sum(np.einsum('ab,...eb->...ea', mats[c], a[..., c::r, :]) for c in range(r))
    return np.moveaxis(out, (-2, -1), (ax_e, ax_n))


class Transfer:
    """Transfers between a coarse level and the next finer level."""

    def __init__(self, fine, coarse, projection="interp"):
        self.fine, self.coarse = fine, coarse
        self.It, self.Pt, self.Rt = time_transfers(fine.tau, coarse.tau)
        fs, cs = fine.space, coarse.space
        self.dg = hasattr(fs, 'P') and hasattr(cs, 'P')
        if self.dg:
            self.dim = fs.dim
            self.Ix, self.Px, self.Rx = space_transfers(fs.P, cs.P)
            if projection == "l2":           # solution projection in space: L2 instead of embedded
                self.Px = l2_projection(fs.P, cs.P)
            # element ratio per direction: 1 (p-coarsening only) or 2 (2:1 h-coarsening)
            self.ratio = (fs.nex // cs.nex, fs.ney // cs.ney)
            for r, nf, nc in zip(self.ratio, (fs.nex, fs.ney), (cs.nex, cs.ney)):
                if r not in (1, 2) or nf != r * nc:
                    raise ValueError("levels must have equal or 2:1 element grids")
            if self.ratio != (1, 1):
                Ih, Ph, Rh = h_transfers(fs.P, cs.P, projection)
                self.hmats = {}
                for d, r in enumerate(self.ratio):
                    self.hmats[d] = ({'I': Ih, 'P': Ph, 'R': Rh} if r == 2 else
                                     {'I': [self.Ix], 'P': [self.Px], 'R': [self.Rx]})

    def _space(self, which, u):
        if not self.dg:
            return u
        if self.ratio != (1, 1):             # u[comp, ey, ex, j, i]: x then y
            c2f = which == 'I'
            out = _apply_dir(self.hmats[0][which], u, 2, 4, c2f)
            if self.dim == 2:
                out = _apply_dir(self.hmats[1][which], out, 1, 3, c2f)
            return out
        mat = {'I': self.Ix, 'P': self.Px, 'R': self.Rx}[which]
        return _apply_space(mat, u, self.dim)

    def project_space(self, u):
        return self._space('P', u)

    def interp(self, Uc):
        """I (coarse -> fine), solution or correction."""
        S = np.stack([self._space('I', Uc[n]) for n in range(Uc.shape[0])])
        return np.tensordot(self.It, S, axes=(1, 0))

    def project(self, Uf):
        """P (fine -> coarse) solution projection."""
        S = np.tensordot(self.Pt, Uf, axes=(1, 0))
        return np.stack([self._space('P', S[n]) for n in range(S.shape[0])])

    def restrict(self, Rf):
        """R = I^T (fine -> coarse) residual restriction."""
        S = np.tensordot(self.Rt, Rf, axes=(1, 0))
        return np.stack([self._space('R', S[n]) for n in range(S.shape[0])])


class MLSDC:
    """Levels ordered coarse (index 0, paper l = 1) to fine (index L-1)."""

    def __init__(self, levels, stages=2, Nc=2, projection="interp", fmg_cycles=1, form="incremental"):
        self.levels = list(levels)
        self.L = len(self.levels)
        self.stages = stages
        self.Nc = Nc
        self.fmg_cycles = fmg_cycles
        self.form = form            # "incremental" (node-to-node) or "zero_to_node"
        self.F = F0n if form == "zero_to_node" else Fnn
        self.T = [Transfer(self.levels[l + 1], self.levels[l], projection) for l in range(self.L - 1)]
        self.sweeps = [0] * self.L

    def _corr(self, l, u0s, U, g, dt, n):
        self.sweeps[l] += n
        if self.form == "zero_to_node":
            return corrector_0n(self.levels[l], u0s[l], U, g, dt, self.stages, n)
        return corrector(self.levels[l], u0s[l], U, g, dt, self.stages, n)

    def initial_values(self, u0):
        u0s = [None] * self.L
        u0s[-1] = u0
        for l in range(self.L - 1, 0, -1):
            u0s[l - 1] = self.T[l - 1].project_space(u0s[l])
        return u0s

    def vcycle(self, u0s, Us, dt, top=None, Nc=None):
        """Algorithm 2 on levels 0..top-1 (top defaults to all levels)."""
        top = self.L if top is None else top
        Nc = self.Nc if Nc is None else Nc
        g = [None] * top
        v = [None] * top
        for l in range(top - 1, 0, -1):
            Us[l] = self._corr(l, u0s, Us[l], g[l], dt, 1)              # pre-sweep
            r = -self.F(self.levels[l], u0s[l], Us[l], dt)                # residual (F^nn or F^0n)
            if g[l] is not None:
                r = r + g[l]
            T = self.T[l - 1]
            v[l - 1] = T.project(Us[l])                                   # solution restriction
            g[l - 1] = self.F(self.levels[l - 1], u0s[l - 1], v[l - 1], dt) + T.restrict(r)
            Us[l - 1] = v[l - 1].copy()
        Us[0] = self._corr(0, u0s, Us[0], g[0], dt, Nc)                  # coarse solve
        for l in range(1, top):
            Us[l] = Us[l] + self.T[l - 1].interp(Us[l - 1] - v[l - 1])  # correction
            if l < top - 1:
                Us[l] = self._corr(l, u0s, Us[l], g[l], dt, 1)           # post-sweep
        return Us

    def start(self, u0s, dt, kind):
        L = self.L
        Us = [None] * L
        if kind in ('cascade', 'fmg1'):
            self.sweeps[0] += 1
            Us[0] = predictor(self.levels[0], u0s[0], dt, self.stages)
            Us[0] = self._corr(0, u0s, Us[0], None, dt, 1)
            if L > 1:
                Us[1] = self.T[0].interp(Us[0])
            for l in range(1, L - 1):
                if kind == 'fmg1':                    # C_fmg V-cycles per added level
                    for _ in range(self.fmg_cycles):
                        self.vcycle(u0s, Us, dt, top=l + 1)
                else:
                    Us[l] = self._corr(l, u0s, Us[l], None, dt, 1)
                Us[l + 1] = self.T[l].interp(Us[l])
        elif kind == 'predictor':
            for l in range(L):
                self.sweeps[l] += 1
                Us[l] = predictor(self.levels[l], u0s[l], dt, self.stages)
        elif kind == 'spread':
            for l in range(L):
                Us[l] = np.stack([u0s[l]] * self.levels[l].M)
        else:
            raise ValueError(kind)
        return Us

    def step(self, u0, dt, ncycles, start='cascade', post_sweep=True, return_levels=False):
        u0s = self.initial_values(u0)
        if self.L == 1:
            # single-level SDC: predictor then ncycles correction sweeps
            self.sweeps[0] += 1
            U = predictor(self.levels[0], u0, dt, self.stages)
            U = self._corr(0, u0s, U, None, dt, ncycles)
            return (U[-1], [U]) if return_levels else U[-1]
        Us = self.start(u0s, dt, start)
        for _ in range(ncycles):
            Us = self.vcycle(u0s, Us, dt)
        if post_sweep:
            Us[-1] = self._corr(self.L - 1, u0s, Us[-1], None, dt, 1)
        return (Us[-1][-1], Us) if return_levels else Us[-1][-1]
