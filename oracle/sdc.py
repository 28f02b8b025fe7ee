"""Single-level SI-SDC building blocks, FP64 (test infrastructure only).

A ``Level`` pairs a spatial problem (``DGSpace`` or the scalar Dahlquist
mode) with a collocation node set.  The spatial problem supplies

    conv(u)      convective part c(u) = -d_x f_c(u)
    diff(u)      physical diffusion part of f (nu L u)
    lap(u)       the scalar diffusion operator L
    nu_d         physical diffusion coefficient entering nu_tilde
    lam_max(u)   max spectral radius of the convective Jacobian
    solve(c, rhs, x0)  solution of (I - c L) x = rhs

and f(u) = conv(u) + diff(u) (Sec. 2, f = -d_x f_c + d_x f_d).

SI operator (Sec. 3.3, eq. H_SI(1)):
    H(u_a, u_b, u_c, dt_m) = dt_m [ c(u_a) + nu_tilde(u_b) L u_c ],
    nu_tilde(u_b) = nu_d + dt_m / 2 * lam_max(u_b)^2
(plus c_s h / P * lam_max(u_b) with artificial viscosity, oracle.av).
Predictors SI(1)/SI(2) (eqs. sdc:incremental_predictor_si1/_si2), the
incremental corrector with Delta H for SI(1)/SI(2) (eqs. DeltaH_SI1,
DeltaH_SI2) plus the FAS term g (Sec. 4.3, eq. ml-sdc:incremental;
Algorithm 1) and the residual F^nn (eq. cm:incremental:op).

Reading: g_m is added to both SI(2) stages (the single-level stage formula
has no g).  Warm starts: stage 1 from u^{k-1}_m, stage 2 from u^(1).
The old terms H(u^{k-1}...) are recomputed here from the stored previous
iterate (the CUDA path caches them, Sec. 3.3 implementation remark).
"""
import numpy as np

from .tables import collocation_nodes, wnn, substeps, c0n


class Level:
    def __init__(self, space, node_kind, M):
        self.space = space
        self.M = int(M)
        self.node_kind = node_kind
        self.tau = collocation_nodes(node_kind, M)
        self.Wnn = wnn(self.tau)
        self.W0n = c0n(self.M) @ self.Wnn          # zero-to-node weights (eq. 0n_weights)
        self.dtau = substeps(self.tau)


def nutilde(space, u_b, dtm):
    # a space may carry a fixed nu_tilde (the library's sisdc_problem.nu_tilde
    # option); the collocation limit does not depend on it (Sec. 3.3: the
    # Delta H terms vanish at convergence)
    fix = getattr(space, "nu_tilde_fix", 0.0)
    if fix > 0.0:
        return fix
    lam = space.lam_max(u_b)
    return space.nu_d + getattr(space, "av_nu_lam", 0.0) * lam + 0.5 * dtm * lam ** 2


def f_eval(space, u):
    return space.conv(u) + space.diff(u)


def quadrature(level, dt, F):
    """Q_m = dt * sum_i w^nn_{m,i} F_i for all m (the S.F product)."""
    return dt * np.tensordot(level.Wnn, F, axes=(1, 0))


def Fnn(level, u0, U, dt):
    """F^nn_m(U) = U_m - U_{m-1} - dt sum_i w^nn_{m,i} f(U_i), U_0 = u0."""
    sp = level.space
    F = np.stack([f_eval(sp, U[i]) for i in range(level.M)])
    Q = quadrature(level, dt, F)
    prev = np.concatenate([u0[None], U[:-1]], axis=0)
    return U - prev - Q


def predictor(level, u0, dt, stages):
    """SI(1) (stages=1) or SI(2) (stages=2) predictor sweep."""
    sp = level.space
    U = np.empty((level.M,) + np.shape(u0), dtype=np.result_type(u0, float))
    uprev = u0
    for m in range(level.M):
        dtm = dt * level.dtau[m]
        if dtm == 0.0:                      # Lobatto t_1 = t_0
            U[m] = uprev
            continue
        cimp = dtm * nutilde(sp, uprev, dtm)
        x1 = sp.solve(cimp, uprev + dtm * sp.conv(uprev), uprev)
        if stages == 2:
            x1 = sp.solve(cimp, uprev + dtm * sp.conv(x1), x1)
        U[m] = x1
        uprev = U[m]
    return U


def corrector(level, u0, U, g, dt, stages, nsweeps):
    """``nsweeps`` incremental SI-MLSDC correction sweeps (Algorithm 1)."""
    sp = level.space
    for _ in range(nsweeps):
        Uold = np.array(U, copy=True)
        Q = quadrature(level, dt, np.stack([f_eval(sp, Uold[i]) for i in range(level.M)]))
        Unew = np.empty_like(Uold)
        unew_prev = u0
        for m in range(level.M):
            dtm = dt * level.dtau[m]
            uold_prev = u0 if m == 0 else Uold[m - 1]
            base = unew_prev + Q[m]
            if g is not None:
                base = base + g[m]
            if dtm == 0.0:                  # Lobatto t_1 = t_0: H terms vanish
                Unew[m] = base
                unew_prev = Unew[m]
                continue
            nu_new = nutilde(sp, unew_prev, dtm)
            nu_old = nutilde(sp, uold_prev, dtm)
            LUold = sp.lap(Uold[m])
            # H(u^{k-1}_{m-1}, u^{k-1}_{m-1}, u^{k-1}_m)
            old1 = dtm * (sp.conv(uold_prev) + nu_old * LUold)
            x1 = sp.solve(dtm * nu_new, base + dtm * sp.conv(unew_prev) - old1, Uold[m])
            if stages == 2:
                # H(u^{k-1}_m, u^{k-1}_{m-1}, u^{k-1}_m)
                old2 = dtm * (sp.conv(Uold[m]) + nu_old * LUold)
                x1 = sp.solve(dtm * nu_new, base + dtm * sp.conv(x1) - old2, x1)
            Unew[m] = x1
            unew_prev = Unew[m]
        U = Unew
    return U


# --------------------------------------------------------------------------
# Non-incremental (zero-to-node) form (Sec. 3.2 "Non-incremental SDC method",
# Sec. 4.5 "Non-incremental multilevel SDC method")
# --------------------------------------------------------------------------
def F0n(level, u0, U, dt):
    """F^0n_m(U) = U_m - u_0 - dt sum_i w^0n_{m,i} f(U_i)."""
    sp = level.space
    F = np.stack([f_eval(sp, U[i]) for i in range(level.M)])
    return U - u0[None] - dt * np.tensordot(level.W0n, F, axes=(1, 0))


def corrector_0n(level, u0, U, g, dt, stages, nsweeps):
    """``nsweeps`` non-incremental SI sweeps: u^k_m = u_0 + dt sum_i w^0n_{m,i}
    f(u^{k-1}_i) + g_m + sum_{i<=m} Delta H^k_i, with the same deltas as the
    incremental sweep, summed over the current and all preceding nodes (g is
    the zero-to-node FAS right-hand side)."""
    sp = level.space
    for _ in range(nsweeps):
        Uold = np.array(U, copy=True)
        Q0 = dt * np.tensordot(level.W0n, np.stack([f_eval(sp, Uold[i]) for i in range(level.M)]), axes=(1, 0))
        Unew = np.empty_like(Uold)
        dH = np.zeros_like(u0)                     # sum of the deltas of the preceding nodes
        unew_prev = u0
        for m in range(level.M):
            dtm = dt * level.dtau[m]
            uold_prev = u0 if m == 0 else Uold[m - 1]
            base = u0 + Q0[m] + dH
            if g is not None:
                base = base + g[m]
            if dtm == 0.0:
                Unew[m] = base
                unew_prev = Unew[m]
                continue
            nu_new = nutilde(sp, unew_prev, dtm)
            nu_old = nutilde(sp, uold_prev, dtm)
            LUold = sp.lap(Uold[m])
            old1 = dtm * (sp.conv(uold_prev) + nu_old * LUold)
            new_expl = dtm * sp.conv(unew_prev)
            x1 = sp.solve(dtm * nu_new, base + new_expl - old1, Uold[m])
            delta = new_expl + dtm * nu_new * sp.lap(x1) - old1
            if stages == 2:
                old2 = dtm * (sp.conv(Uold[m]) + nu_old * LUold)
                new_expl = dtm * sp.conv(x1)
                x1 = sp.solve(dtm * nu_new, base + new_expl - old2, x1)
                delta = new_expl + dtm * nu_new * sp.lap(x1) - old2
            Unew[m] = x1
            dH = dH + delta
            unew_prev = Unew[m]
        U = Unew
    return U
