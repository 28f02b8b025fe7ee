"""Pins for the oracle's SI-SDC / SI-MLSDC algorithms (CPU only).

* Dahlquist problem (Sec. 5): the SI(1) predictor equals its closed-form
  substep product; sweeps and V-cycles converge to the collocation stability
  function, which equals the textbook Pade approximant of e^z
  ((M-1, M) for Radau IIA, (M-1, M-1) for Lobatto IIIA).
* PDE: SDC and MLSDC iterates converge to the dense brute-force collocation
  solution (I - dt W^0n (x) A_h) U = 1 (x) u_0; a V-cycle started at the
  collocation solution leaves it unchanged (FAS fixed point); the converged
  result does not depend on nu_tilde; mass is conserved; the 1D
  convection-diffusion step matches the exact damped, shifted modes.
"""
import math

import numpy as np
import pytest

from oracle import sdc as S
from oracle.dahlquist import stability, DahlquistSpace
from oracle.dg import DGSpace, ConvDiff, Burgers2
from oracle.mlsdc import MLSDC
from oracle.sdc import Level
from oracle.tables import collocation_nodes, w0n
from paper_2504_18526_gb300 import inputs


def pade_exp(k, m, z):
    num = sum(math.factorial(k + m - j) * math.factorial(k) /
              (math.factorial(k + m) * math.factorial(j) * math.factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(math.factorial(k + m - j) * math.factorial(m) /
              (math.factorial(k + m) * math.factorial(j) * math.factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


ZS = [-0.7 + 1.3j, -3.0 + 0.5j, -0.1 + 2.0j, -8.0 + 0.0j]


@pytest.mark.parametrize("z", ZS)
def test_si1_predictor_closed_form(z):
    for kind, M in [("radau_right", 3), ("radau_right", 5), ("lobatto", 4)]:
        dtau = np.diff(np.concatenate([[0.0], collocation_nodes(kind, M)]))
        R = 1.0
        for d in dtau:
            zr, zi = (d * z).real, (d * z).imag
            R *= (1 + 1j * zi) / (1 - zr + zi * zi / 2)
        sp = DahlquistSpace(z)
        U = S.predictor(Level(sp, kind, M), np.complex128(1.0), 1.0, stages=1)
        assert abs(U[-1] - R) < 1e-14


@pytest.mark.parametrize("z", ZS)
@pytest.mark.parametrize("kind,Ms", [("radau_right", [3, 5]), ("radau_right", [3, 5, 7]),
                                     ("lobatto", [3, 5]), ("lobatto", [2, 3, 5])])
def test_collocation_limit_is_pade(z, kind, Ms):
    M = Ms[-1]
    pade = pade_exp(M - 1, M, z) if kind == "radau_right" else pade_exp(M - 1, M - 1, z)
    for stages in (1, 2):
        assert abs(stability(z, [M], kind, stages, ncycles=40) - pade) < 1e-12
        start = "fmg1" if len(Ms) > 2 else "cascade"
        assert abs(stability(z, Ms, kind, stages, ncycles=30, start=start) - pade) < 1e-12
        assert abs(stability(z, Ms, kind, stages, ncycles=30, start="predictor") - pade) < 1e-12


@pytest.mark.parametrize("kind,M,order", [("radau_right", 2, 3), ("radau_right", 3, 5),
                                           ("lobatto", 3, 4), ("lobatto", 4, 6)])
def test_converged_order_radau_2m_minus_1_lobatto_2m_minus_2(kind, M, order):
    """At convergence the SDC step is the collocation method, of order 2M-1
    on Radau-Right nodes (Radau IIA) and 2M-2 on Lobatto nodes (Lobatto
    IIIA) (Sec. 3.3): the one-step error |R(z) - e^z| scales as |z|^(p+1)."""
    z0 = -0.6 + 0.8j
    errs = []
    for h in (0.4, 0.2):
        z = h * z0
        errs.append(abs(stability(z, [M], kind, 2, ncycles=60) - np.exp(z)))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - (order + 1)) < 0.35


@pytest.mark.parametrize("stages", [1, 2])
@pytest.mark.parametrize("M,sweeps", [(3, 1), (3, 4), (5, 2), (5, 8)])
def test_radau_si_sdc_l_stable(stages, M, sweeps):
    """L-stability of the SI-SDC step on Radau-Right nodes for any number of
    sweeps (the property the paper cites for SI-SDC): as the stiff implicit
    part grows, Re z -> -inf with the explicit part fixed, every iterate is
    O(1/|z|), so R(z) -> 0."""
    r = [abs(stability(-x + 2.0j, [M], "radau_right", stages, ncycles=sweeps)) for x in (1e8, 1e9)]
    assert r[1] < 1e-7
    assert 5.0 < r[0] / r[1] < 20.0          # decays like 1/|z|


def test_mlsdc_fewer_cycles_than_sdc_sweeps():
    """MLSDC reaches a given accuracy in fewer fine sweeps (Sec. 5.2, Sec. 7)."""
    z = -2.0 + 4.0j
    pade = pade_exp(6, 7, z)
    def first_below(fn, eps=1e-10):
        for n in range(1, 60):
            if abs(fn(n) - pade) < eps:
                return n
        return 99
    n_sdc = first_below(lambda n: stability(z, [7], "radau_right", 2, ncycles=n))
    n_ml = first_below(lambda n: stability(z, [3, 5, 7], "radau_right", 2, ncycles=n - 1,
                                           start="fmg1"))
    assert n_ml < n_sdc


# ---------------------------------------------------------------------------
# PDE brute force on a tiny 1D convection-diffusion mesh
# ---------------------------------------------------------------------------
def _tiny_problem(P=4, nel=5, nu=0.05, a=1.0):
    pde = ConvDiff((a, 0.0), nu)
    return lambda p: DGSpace(1, (nel,), p, (0.0, 0.0), (2 * math.pi, 0.0), pde, cg_rtol=1e-15)


def _dense_f(sp):
    n = int(np.prod(sp.shape))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = S.f_eval(sp, e.reshape(sp.shape)).ravel()
    return A


def _collocation(sp, kind, M, u0, dt):
    Ah = _dense_f(sp)
    W = w0n(collocation_nodes(kind, M))
    n = Ah.shape[0]
    big = np.eye(M * n) - dt * np.kron(W, Ah)
    U = np.linalg.solve(big, np.tile(u0.ravel(), M))
    return U.reshape((M,) + sp.shape)


@pytest.mark.parametrize("kind", ["radau_right", "lobatto"])
def test_pde_converges_to_collocation(kind):
    mk = _tiny_problem()
    fine = mk(4)
    X, _ = fine.coords()
    u0 = np.sin(X)[None] + 0.3 * np.cos(2 * X)[None]
    dt = 0.2
    Uc = _collocation(fine, kind, 5, u0, dt)
    for stages in (1, 2):
        # single-level SDC
        ml1 = MLSDC([Level(fine, kind, 5)], stages=stages)
        _, [U] = ml1.step(u0, dt, 45, return_levels=True)
        assert np.max(np.abs(U - Uc)) < 1e-11
        # two-level MLSDC with space and time coarsening
        ml = MLSDC([Level(mk(2), kind, 3), Level(fine, kind, 5)], stages=stages)
        errs = []
        for nc in (2, 10, 45):
            _, Us = ml.step(u0, dt, nc, start="cascade", return_levels=True)
            errs.append(np.max(np.abs(Us[-1] - Uc)))
        assert errs[-1] < 1e-11 and errs[0] > errs[1] > errs[2]
        # every level converges to the fine solution (the FAS right-hand side at
        # work): the coarse iterate is the projection of the fine collocation
        # solution, not the coarse level's own collocation solution
        Pc = ml.T[0].project(Uc)
        assert np.max(np.abs(Us[0] - Pc)) < 1e-11
        own = _collocation(mk(2), kind, 3, ml.T[0].project_space(u0), dt)
        assert np.max(np.abs(own - Pc)) > 1e-6


@pytest.mark.parametrize("projection", ["interp", "l2"])
def test_fas_fixed_point(projection):
    """A V-cycle started at the collocation solution leaves it unchanged,
    whichever solution projection the FAS right-hand side uses."""
    mk = _tiny_problem()
    kind = "radau_right"
    fine, coarse = mk(4), mk(2)
    X, _ = fine.coords()
    u0 = np.sin(X)[None]
    dt = 0.3
    Uc = _collocation(fine, kind, 5, u0, dt)
    ml = MLSDC([Level(coarse, kind, 3), Level(fine, kind, 5)], stages=2, projection=projection)
    u0s = ml.initial_values(u0)
    Us = [np.zeros((3,) + coarse.shape), Uc.copy()]
    ml.vcycle(u0s, Us, dt)
    assert np.max(np.abs(Us[-1] - Uc)) < 1e-13


def test_converged_result_independent_of_nutilde(monkeypatch):
    mk = _tiny_problem()
    fine = mk(4)
    X, _ = fine.coords()
    u0 = np.sin(X)[None]
    ml = MLSDC([Level(mk(2), "radau_right", 3), Level(fine, "radau_right", 5)], stages=2)
    ref = ml.step(u0, 0.2, 45)
    orig = S.nutilde
    monkeypatch.setattr(S, "nutilde", lambda sp, ub, dtm: 2.0 * orig(sp, ub, dtm))
    alt = ml.step(u0, 0.2, 45)
    assert np.max(np.abs(alt - ref)) < 1e-11
    few_ref = ml.step(u0, 0.2, 1)
    monkeypatch.setattr(S, "nutilde", orig)
    assert np.max(np.abs(few_ref - ml.step(u0, 0.2, 1))) > 1e-8   # nu_tilde does act


def test_fixed_nutilde_option_same_collocation_limit():
    """A space carrying a fixed nu_tilde (the option the library exposes as
    sisdc_problem.nu_tilde) converges to the same collocation solution as the
    method's nu_d + dt_m/2 lam_max^2, and with few sweeps it does act."""
    mk = _tiny_problem()
    X, _ = mk(4).coords()
    u0 = np.sin(X)[None]

    def run(ncyc, fix):
        levels = [Level(mk(2), "radau_right", 3), Level(mk(4), "radau_right", 5)]
        for lv in levels:
            lv.space.nu_tilde_fix = fix
        return MLSDC(levels, stages=2).step(u0, 0.2, ncyc)

    assert np.max(np.abs(run(45, 0.1) - run(45, 0.0))) < 1e-12
    assert np.max(np.abs(run(1, 0.1) - run(1, 0.0))) > 1e-8


def test_mass_conservation_burgers_step():
    pde = Burgers2(5e-3)
    mk = lambda p: DGSpace(2, (4, 4), p, (0.0, 0.0), (1.0, 1.0), pde, cg_rtol=1e-15)
    fine = mk(5)
    X, Y = fine.coords()
    u0 = inputs.burgers2d_initial(X, Y)
    ml = MLSDC([Level(mk(3), "radau_right", 3), Level(fine, "radau_right", 5)], stages=2)
    u1 = ml.step(u0, 2e-3, 2)
    assert np.max(np.abs(fine.integral(u1) - fine.integral(u0))) < 1e-13


def test_convdiff1d_exact_solution():
    """Config convdiff1d: 40 steps to t = 2 against the exact solution; the
    error drops at high order when the mesh and step are refined."""
    w = inputs.WORKLOADS["convdiff1d"]
    pde = ConvDiff(w["adv"], w["nu"])
    errs = []
    for nel, P, dt, nsteps in [(16, 4, 0.05, 40), (32, 4, 0.025, 80)]:
        mk = lambda p: DGSpace(1, (nel,), p, w["lo"], w["hi"], pde, cg_rtol=1e-13)
        fine = mk(P)
        X, _ = fine.coords()
        u = inputs.convdiff1d_exact(X, 0.0)
        ml = MLSDC([Level(mk(2), w["nodes"], 3), Level(fine, w["nodes"], 5)], stages=2)
        for n in range(nsteps):
            u = ml.step(u, dt, w["ncycles"])
        errs.append(fine.l2(u - inputs.convdiff1d_exact(X, nsteps * dt)))
    assert errs[0] < 2e-4
    assert errs[0] / errs[1] > 16.0        # at least 4th order under joint refinement


def test_ns_step_conserves_mass_momentum_energy():
    """Shear-layer data on a coarse grid: one two-level SI-MLSDC step conserves
    all four integrals to round-off (conservative convective, viscous and SIPG
    operators on a periodic mesh) and changes the state."""
    from oracle.dg import NavierStokes2
    w = inputs.WORKLOADS["ns_shear"]
    pde = NavierStokes2(w["gamma"], 200.0, w["Pr"])
    mk = lambda p: DGSpace(2, (4, 4), p, (0.0, 0.0), (1.0, 1.0), pde, cg_rtol=1e-15)
    fine = mk(4)
    X, Y = fine.coords()
    u0 = inputs.shear_layer(X, Y, w["gamma"], w["mach"], delta=0.1)
    ml = MLSDC([Level(mk(2), "radau_right", 3), Level(fine, "radau_right", 5)], stages=2)
    u1 = ml.step(u0, 2e-4, 2)
    scale = np.max(np.abs(fine.integral(u0))) + 1.0
    assert np.max(np.abs(fine.integral(u1) - fine.integral(u0))) < 1e-13 * scale
    assert np.max(np.abs(u1 - u0)) > 1e-6


@pytest.mark.parametrize("test", ["test1", "test2"])
def test_paper_wave_packet_iteration_counts(test):
    """The paper's preliminary 1D studies: single-level SDC and the three-level
    V-cycle reach convergence after the printed numbers of sweeps / cycles
    (test 1 exactly; test 2 within one cycle for MLSDC)."""
    from tests.helpers import wave_packet_fixture, wave_packet_exact, converged_at
    coef, tests = wave_packet_fixture()
    Ms, sdc_sweeps, ml_cycles = tests[test]
    nu, v, dt = 2e-2, 1.0, 1e-2

    def exact(X, t):
        return wave_packet_exact(coef, X, t, nu, v)

    mk = lambda: DGSpace(1, (32,), 15, (0.0, 0.0), (1.0, 0.0), ConvDiff((v, 0.0), nu), cg_rtol=1e-14,
                         cg_maxit=10000)
    fine = mk()
    X, _ = fine.coords()
    u0, ue = exact(X, 0.0), exact(X, dt)
    levels = [Level(mk(), "radau_right", M) for M in Ms]
    # single-level SDC on the finest level: the predictor counts as the first sweep
    U = S.predictor(levels[-1], u0, dt, 2)
    errs = [fine.l2(U[-1] - ue)]
    for _ in range(sdc_sweeps + 4):
        U = S.corrector(levels[-1], u0, U, None, dt, 2, 1)
        errs.append(fine.l2(U[-1] - ue))
    assert converged_at(errs) + 1 == sdc_sweeps
    ml = MLSDC(levels, stages=2, Nc=2)
    u0s = ml.initial_values(u0)
    Us = ml.start(u0s, dt, "predictor")
    errm = [fine.l2(Us[-1][-1] - ue)]
    for _ in range(ml_cycles + 4):
        Us = ml.vcycle(u0s, Us, dt)
        errm.append(fine.l2(Us[-1][-1] - ue))
    got = converged_at(errm)
    if test == "test1":
        assert got == ml_cycles
    else:
        assert abs(got - ml_cycles) <= 1
    assert errm[got] < 1e-10     # converged to the collocation error, far below the start


@pytest.mark.parametrize("projection", ["interp", "l2"])
def test_fmg_start_with_several_cycles_converges(projection):
    """Three levels, FMG start with C_fmg = 2 V-cycles per added level: the
    step converges to the fine collocation solution as cycles are added, and
    C_fmg = 2 starts closer than C_fmg = 1."""
    mk = _tiny_problem()
    kind = "radau_right"
    fine = mk(5)
    X, _ = fine.coords()
    u0 = np.sin(X)[None]
    dt = 0.3
    Uc = _collocation(fine, kind, 5, u0, dt)
    errs = {}
    for C in (1, 2):
        ml = MLSDC([Level(mk(2), kind, 2), Level(mk(3), kind, 3), Level(fine, kind, 5)], stages=2,
                   projection=projection, fmg_cycles=C)
        u0s = ml.initial_values(u0)
        Us = ml.start(u0s, dt, "fmg1")
        errs[C] = [np.max(np.abs(Us[-1] - Uc))]
        for _ in range(30):
            Us = ml.vcycle(u0s, Us, dt)
            errs[C].append(np.max(np.abs(Us[-1] - Uc)))
    assert errs[2][0] < errs[1][0]
    assert errs[1][-1] < 1e-9 and errs[2][-1] < 1e-9


def test_non_incremental_sdc_equals_incremental_single_level():
    """Single level: the zero-to-node sweeps give the incremental iterates
    (the same deltas summed over the preceding nodes)."""
    mk = _tiny_problem()
    fine = mk(4)
    X, _ = fine.coords()
    u0 = np.sin(X)[None]
    for kind in ("radau_right", "lobatto"):
        for stages in (1, 2):
            L = Level(fine, kind, 5)
            U = S.predictor(L, u0, 0.3, stages)
            a = S.corrector(L, u0, U, None, 0.3, stages, 3)
            b = S.corrector_0n(L, u0, U, None, 0.3, stages, 3)
            assert np.max(np.abs(a - b)) < 1e-13


def test_non_incremental_mlsdc_converges_and_differs():
    """Two levels: the zero-to-node MLSDC has the collocation solution as its
    FAS fixed point and converges to it, but its iterates differ from the
    incremental MLSDC (the forms are not equivalent, Sec. 4.6)."""
    mk = _tiny_problem()
    kind = "radau_right"
    fine = mk(4)
    X, _ = fine.coords()
    u0 = np.sin(X)[None]
    dt = 0.3
    Uc = _collocation(fine, kind, 5, u0, dt)
    ml = {f: MLSDC([Level(mk(2), kind, 3), Level(fine, kind, 5)], stages=2, form=f)
          for f in ("incremental", "zero_to_node")}
    u0s = ml["zero_to_node"].initial_values(u0)
    Us = [np.zeros((3,) + mk(2).shape), Uc.copy()]
    ml["zero_to_node"].vcycle(u0s, Us, dt)
    assert np.max(np.abs(Us[-1] - Uc)) < 1e-13
    one = {f: ml[f].step(u0, dt, 1, start="predictor") for f in ml}
    assert np.max(np.abs(one["zero_to_node"] - one["incremental"])) > 1e-8
    conv = ml["zero_to_node"].step(u0, dt, 40, start="predictor")
    assert np.max(np.abs(conv - Uc[-1])) < 1e-10
