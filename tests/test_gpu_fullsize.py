"""The 2D workloads at their stated sizes against the CPU oracle, and the
Euler vortex against its exact solution under h-refinement.

* Euler isentropic vortex, 64 x 64 elements, P = 7/5/3, Lobatto 5/3/2, FMG1
  start, 3 V-cycles: two steps in the launch configuration the bench times
  (CUDA graph, autotuned tile shapes), FP64, within 1e-12 of the oracle.
* Navier-Stokes shear layer, 128 x 128 elements, P = 5/3, Radau-Right 5/3,
  Cascade start, 3 V-cycles: one step, FP64, within 1e-12 of the oracle.
* Euler vortex over one full period (the vortex returns to its start on the
  periodic box, Sec. 2 problem statement with the standard vortex data) on
  16^2 and 32^2 elements with the workload's degrees and nodes at CFL 0.5:
  the error against the exact solution falls at about the rate P + 1 of the
  fine degree under h-refinement (time step refined with h).

Both sides solve the implicit systems to rtol 1e-14 in the parity cases.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S   # noqa: E402
from tests.helpers import oracle_ml, rel_l2              # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def _coords(ctx, w):
    nc, n, M = ctx.info(-1)
    hx, hy = np.zeros(n), np.zeros(n)
    S.sisdc_level_coords(ctx.levels[-1], hx, hy)
    lv = w["levels"][-1]
    shp = (lv["nel"][1], lv["nel"][0], lv["P"] + 1, lv["P"] + 1)
    return hx.reshape(shp), hy.reshape(shp)


def _parity(w, name, nsteps, dev):
    ctx = S.Context(w, cg_rtol=1e-14, cg_maxit=10000, use_graph=1)
    X, Y = _coords(ctx, w)
    u0 = inputs.initial_state(name, X, Y)
    lv = w["levels"][-1]
    dt = inputs.cfl_dt(w["cfl"], (w["hi"][0] - w["lo"][0]) / lv["nel"][0], lv["P"],
                       inputs.max_wave_speed(w["pde"], u0, w.get("gamma", 1.4)))
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    S.sisdc_autotune(ctx.ctx, du, dt, len(w["levels"]))
    om = oracle_ml(w)
    u = u0
    worst = 0.0
    for n in range(nsteps):
        u = om.step(u, dt, w["ncycles"], start=w["start"])
        S.sisdc_step(ctx.ctx, du, n * dt, dt, w["ncycles"], S.START_IDS[w["start"]], 1)
        torch.cuda.synchronize()
        worst = max(worst, rel_l2(du.cpu().numpy(), u))
    S.sisdc_sync(ctx.ctx)
    ctx.close()
    return worst, float(np.max(np.abs(u - u0)))


def test_step_parity_euler_vortex_full_size(dev):
    w = inputs.WORKLOADS["euler_vortex"]
    worst, moved = _parity(w, "euler_vortex", 2, dev)
    print("euler_vortex 64^2: worst step rel L2 vs oracle %.3e" % worst)
    assert worst < TOL and moved > 1e-6


def test_step_parity_ns_shear_full_size(dev):
    w = inputs.WORKLOADS["ns_shear"]
    worst, moved = _parity(w, "ns_shear", 1, dev)
    print("ns_shear 128^2: step rel L2 vs oracle %.3e" % worst)
    assert worst < TOL and moved > 1e-6


def _vortex_period_error(nel, dev):
    """GLL-quadrature L2 error (all four variables) after one period on an
    nel x nel mesh, relative to the L2 norm of the initial perturbation of
    the free stream."""
    w = inputs.scaled("euler_vortex", nel=(nel, nel))
    ctx = S.Context(w, cg_rtol=1e-12, cg_maxit=10000, use_graph=1)
    X, Y = _coords(ctx, w)
    u0 = inputs.initial_state("euler_vortex", X, Y)
    lv = w["levels"][-1]
    h = (w["hi"][0] - w["lo"][0]) / nel
    dt_cfl = inputs.cfl_dt(w["cfl"], h, lv["P"], inputs.max_wave_speed("euler", u0))
    vinf = w["mach"] * math.sqrt(w["gamma"])
    period = (w["hi"][0] - w["lo"][0]) / (vinf * math.cos(math.radians(w["angle_deg"])))
    nsteps = int(math.ceil(period / dt_cfl))
    dt = period / nsteps
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    ref = torch.from_numpy(np.ascontiguousarray(inputs.isentropic_vortex(X, Y, period))).to(dev)
    free = torch.from_numpy(np.ascontiguousarray(inputs.isentropic_vortex(X, Y, 0.0, beta=0.0))).to(dev)
    for n in range(nsteps):
        S.sisdc_step(ctx.ctx, du, n * dt, dt, w["ncycles"], S.START_IDS[w["start"]], 1)
    S.sisdc_sync(ctx.ctx)
    err = S.sisdc_norms(ctx.levels[-1], du, ref)[0]
    size = S.sisdc_norms(ctx.levels[-1], ref, free)[0]
    ctx.close()
    return float(np.sqrt(np.sum(err ** 2)) / np.sqrt(np.sum(size ** 2))), nsteps


def test_euler_vortex_one_period_h_convergence(dev):
    e16, n16 = _vortex_period_error(16, dev)
    e32, n32 = _vortex_period_error(32, dev)
    rate = math.log2(e16 / e32)
    print("euler vortex, one period (t = 47.81): 16^2 %d steps rel L2 error %.3e; 32^2 %d steps %.3e; rate %.2f"
          % (n16, e16, n32, e32, rate))
    assert e32 < e16 < 1e-2
    assert rate > 5.0
