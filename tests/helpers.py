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
    return DGSpace(w["dim"], tuple(lvl["nel"][:w["dim"]]), lvl["P"], w["lo"], w["hi"],
                   oracle_pde(w), cg_rtol=rtol, cg_maxit=10000)


def oracle_ml(w, stages=2, Nc=2, rtol=1e-14):
    levels = [Level(oracle_space(w, lv, rtol), w["nodes"], lv["M"]) for lv in w["levels"]]
    return MLSDC(levels, stages=stages, Nc=Nc)


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
