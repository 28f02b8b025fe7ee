"""Artificial viscosity (Persson-Peraire, Sec. 6; the shock-capturing
workloads of Sec. 8) on the GPU against the CPU oracle, through the C ABI:
f with the viscosity term, whole MLSDC steps with 2:1 h-coarsening (the
Burgers moving front) and p-coarsening (Sod's shock tube), the full-size Sod
set-up, and Sod's solution after 32 steps against the exact Riemann
solution."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S   # noqa: E402
from oracle import av as OAV                              # noqa: E402
from oracle import sdc as OS                              # noqa: E402
from tests.helpers import oracle_ml, oracle_space, rel_l2   # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def T(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def N(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def make_ctx(w, rtol=1e-14, **kw):
    return S.Context(w, cg_rtol=rtol, cg_maxit=10000, **kw)


CASES = {
    "burgers": dict(pde="burgers", dim=2, ncomp=2, nu=1e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
                    levels=[dict(nel=(6, 4), P=3, M=3), dict(nel=(6, 4), P=6, M=5)],
                    av=dict(kappa=0.5, cs=0.5, comp=0)),
    "euler": dict(pde="euler", dim=2, ncomp=4, gamma=1.4, lo=(0.0, 0.0), hi=(2.0, 1.0), nodes="radau_right",
                  levels=[dict(nel=(8, 3), P=2, M=3), dict(nel=(8, 3), P=5, M=5)],
                  av=dict(kappa=2.0, cs=0.4, comp=0)),
    "convdiff1d": dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=1e-3, lo=(0.0, 0.0), hi=(1.0, 0.0),
                       nodes="radau_right", levels=[dict(nel=(9, 1), P=4, M=3), dict(nel=(9, 1), P=12, M=5)],
                       av=dict(kappa=1.0, cs=0.3, comp=0)),
}


def mixed_state(w, sp, seed):
    """Half of the elements rough (random nodal values: the sensor sees
    energy in the top modes), half smooth (linear in x on
    each element: no top-mode energy, no viscosity); Euler states physical."""
    rng = np.random.default_rng(seed)
    X, _ = sp.coords()
    xi = (X - X.min(axis=(-2, -1), keepdims=True)) / sp.hx
    smooth = 0.3 + 0.2 * xi
    rough = rng.random(sp.shape)
    odd = (np.arange(sp.nex) % 2 == 1)[None, :, None, None]
    if w["pde"] == "euler":
        u = np.empty(sp.shape)
        u[0] = 1.0 + 0.4 * np.where(odd, rough[0], smooth)
        u[1] = 0.3 * np.where(odd, rough[1] - 0.5, smooth)
        u[2] = 0.2 * np.where(odd, rough[2] - 0.5, smooth)
        u[3] = 2.5 + 0.5 * np.where(odd, rough[3], smooth)
        return u
    return np.where(odd[None], rough - 0.5, smooth[None] * np.ones(sp.shape))


@pytest.mark.parametrize("case", sorted(CASES))
def test_apply_f_with_av_parity(dev, case):
    w = CASES[case]
    ctx = make_ctx(w)
    for li, lvl in enumerate(w["levels"]):
        sp = oracle_space(w, lvl)
        u = mixed_state(w, sp, 40 + li)
        eps = OAV.viscosity(sp, u, **w["av"])
        assert eps.max() > 0.0 and eps.min() == 0.0               # both regimes present
        du = T(u, dev)
        out = torch.empty_like(du)
        S.sisdc_apply_f(ctx.levels[li], du, out)
        ref = OS.f_eval(sp, u)
        assert rel_l2(N(out), ref) < TOL, (case, li, rel_l2(N(out), ref))
        sp.av = None
        assert rel_l2(ref, OS.f_eval(sp, u)) > 1e-4                # the viscosity term matters here
    S.sisdc_sync(ctx.ctx)
    ctx.close()


def _front_small():
    w = inputs.scaled("burgers_front", levels=[dict(nel=(4, 1), P=4, M=3), dict(nel=(8, 1), P=4, M=5)])
    return w


def _sod_small():
    return inputs.scaled("sod", levels=[dict(nel=(20, 1), P=2, M=3), dict(nel=(20, 1), P=4, M=5)])


@pytest.mark.parametrize("which", ["front", "sod"])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_step_parity_with_av(dev, which, use_graph):
    """Whole steps (V-cycles with the viscosity on every level) within 1e-12
    of the oracle: the Burgers front with 2:1 h-coarsening and FMG_1, Sod with
    p-coarsening and Cascade."""
    w = _front_small() if which == "front" else _sod_small()
    sp = oracle_space(w, w["levels"][-1])
    X, Y = sp.coords()
    if which == "front":
        u0 = inputs.burgers_front(X, 0.0, w["nu"])
        dt = inputs.cfl_dt(4.0, sp.hx, sp.P, inputs.max_wave_speed("burgers", u0))
    else:
        u0 = inputs.sod_state(X, 0.0)
        dt = w["T"] / 16
    om = oracle_ml(w)
    ctx = make_ctx(w, use_graph=use_graph)
    u = u0.copy()
    du = T(u0, dev)
    active = False
    for n in range(2):
        u = om.step(u, dt, 2, start=w["start"])
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 2, S.START_IDS[w["start"]], 1)
        assert rel_l2(N(du), u) < TOL, (which, n, rel_l2(N(du), u))
        active = active or OAV.viscosity(sp, u, **w["av"]).max() > 0.0
    assert active                                                  # the viscosity was switched on
    S.sisdc_sync(ctx.ctx)
    ctx.close()


def test_sod_full_size_parity(dev):
    """The Sod set-up at its full size (80 elements per unit length, P = 5/3,
    Radau-Right 7/5, Cascade) in the bench's launch configuration (CUDA graph,
    autotuned): two steps of dt = 0.2/32 within 1e-12 of the oracle."""
    w = inputs.WORKLOADS["sod"]
    sp = oracle_space(w, w["levels"][-1])
    X, Y = sp.coords()
    u0 = inputs.sod_state(X, 0.0)
    dt = w["T"] / w["nsteps"]
    om = oracle_ml(w)
    ctx = make_ctx(w, use_graph=1)
    du = T(u0, dev)
    S.sisdc_autotune(ctx.ctx, du, dt, len(w["levels"]))
    u = u0.copy()
    for n in range(2):
        u = om.step(u, dt, 2, start="cascade")
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 2, S.START_IDS["cascade"], 1)
        assert rel_l2(N(du), u) < TOL
    S.sisdc_sync(ctx.ctx)
    ctx.close()


def test_sod_32_steps_against_exact(dev):
    """32 steps of MLSDC (3 V-cycles each) to t = 0.2: density within 5e-3 (L1
    on [0, 1]) of the exact Riemann solution (the oracle reaches 1.95e-3), the
    velocity overshoot at the shock below 15 % of u* (the oracle: 8.9 %), mass
    conserved to round-off (Rusanov, SIPG and the BR1 viscosity are all
    conservative)."""
    w = inputs.WORKLOADS["sod"]
    sp = oracle_space(w, w["levels"][-1])
    X, _ = sp.coords()
    u0 = inputs.sod_state(X, 0.0)
    dt = w["T"] / w["nsteps"]
    ctx = make_ctx(w, rtol=1e-12, use_graph=1)
    du = T(u0, dev)
    for n in range(w["nsteps"]):
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 3, S.START_IDS["cascade"], 1)
    u = N(du).reshape(sp.shape)
    S.sisdc_sync(ctx.ctx)
    ctx.close()
    ex = inputs.sod_state(X, w["T"])
    half = np.broadcast_to(X <= 1.0, X.shape)
    rho_err = np.sum((sp.mass * np.abs(u[0] - ex[0]))[half]) / np.sum(sp.mass[None, None] * half)
    assert np.all(np.isfinite(u))
    assert rho_err < 5e-3, rho_err
    ps, us = inputs._sod_star()
    v = u[1] / u[0]
    assert v[half].max() < 1.15 * us
    m0, m1 = np.sum(sp.mass * u0[0]), np.sum(sp.mass * u[0])
    assert abs(m1 - m0) < 1e-12 * m0


def test_av_api_rules(dev):
    w = CASES["burgers"]
    ctx = S.Context(w)                                   # the workload sets the viscosity first
    with pytest.raises(S.SisdcError):
        S.sisdc_set_av(ctx.ctx, 0.5, 0.5, 0)              # after the first level
    ctx.close()
    plain = dict(w)
    plain.pop("av")
    c2 = S.sisdc_create(S.make_problem(plain), 0)
    with pytest.raises(S.SisdcError):
        S.sisdc_set_av(c2, 0.5, 0.5, 2)                   # Burgers has components 0, 1
    with pytest.raises(S.SisdcError):
        S.sisdc_set_av(c2, 0.0, 0.5, 0)                   # d_s must be positive
    S.sisdc_set_av(c2, 0.5, 0.0, 0)                       # c_s = 0: off
    S.sisdc_destroy(c2)
