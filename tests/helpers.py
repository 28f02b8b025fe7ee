"""Shared test helpers: oracle construction from a workload description and
array plumbing between numpy (oracle) and torch (CUDA library)."""
import numpy as np

from oracle.dg import DGSpace, ConvDiff, Burgers2, Euler2, NavierStokes2
from oracle.mlsdc import MLSDC
from oracle.sdc import Level


def oracle_pde(w):
    if w["pde"] == "convdiff":
        return ConvDiff(w["adv"], w["nu"])
    if w["pde"] == "burgers":
        return Burgers2(w["nu"])
    if w["pde"] == "euler":
        return Euler2(w["gamma"])
    if w["pde"] == "ns":
        return NavierStokes2(w["gamma"], w["Re"], w["Pr"], w.get("rho_ref", 1.0))
    raise ValueError(w["pde"])


def oracle_space(w, lvl, rtol=1e-14):
    sp = DGSpace(w["dim"], tuple(lvl["nel"][:w["dim"]]), lvl["P"], w["lo"], w["hi"],
                 oracle_pde(w), cg_rtol=rtol, cg_maxit=10000)
    if w.get("av"):
        sp.av = dict(w["av"])
    return sp


def oracle_ml(w, stages=2, Nc=2, rtol=1e-14, **kw):
    levels = [Level(oracle_space(w, lv, rtol), w["nodes"], lv["M"]) for lv in w["levels"]]
    return MLSDC(levels, stages=stages, Nc=Nc, **kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=float).ravel()
    b = np.asarray(b, dtype=float).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def physical_euler_state(shape, rng):
    u = np.empty(shape)
    u[0] = 1.0 + 0.3 * rng.random(shape[1:])
    u[1] = 0.4 * rng.standard_normal(shape[1:])
    u[2] = 0.4 * rng.standard_normal(shape[1:])
    u[3] = 2.5 + 0.3 * rng.random(shape[1:])
    return u


def random_state(w, shape, seed):
    rng = np.random.default_rng(1000 + seed)
    if w["pde"] in ("euler", "ns"):
        return physical_euler_state(shape, rng)
    return rng.standard_normal(shape)


def wave_packet_fixture():
    """Coefficients (kappa, a, s) and the printed iteration counts of the
    paper's preliminary 1D studies (tests/golden/wave_packet_iterations.txt)."""
    import math
    import os
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", "wave_packet_iterations.txt"))
            if ln.strip() and not ln.startswith("#")]
    coef = [(float(r[0]) * math.pi, float(r[1]), float(r[2])) for r in rows if not r[0].startswith("test")]
    tests = {r[0]: (tuple(int(m) for m in r[1].split(",")), int(r[2]), int(r[3])) for r in rows if r[0].startswith("test")}
    return coef, tests


def wave_packet_exact(coef, X, t, nu=2e-2, v=1.0):
    """u = sum_i a_i sin(kappa_i (x - s_i - v t)) exp(-kappa_i^2 nu t)."""
    import math
    return sum(a * np.sin(k * (X - s - v * t)) * math.exp(-k * k * nu * t) for k, a, s in coef)[None]


def converged_at(errs):
    """First iteration whose L2 error differs from the previous one by less than 10 %."""
    for k in range(1, len(errs)):
        if abs(errs[k] - errs[k - 1]) <= 0.1 * abs(errs[k - 1]):
            return k
    return None
