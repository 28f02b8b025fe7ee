"""The learned initial guess inside the method (sisdc_set_learned): the fine
level's correction sweeps, composed from the single-operation kernels, add
the network's correction to the warm start of every implicit solve.

* with any network the step's result is the plain method's to the solver
  tolerance: with solves to rtol 1e-14 the learned form matches the CPU
  oracle to 1e-12 per step (2D Burgers, Navier-Stokes);
* a network trained on the plain method's own logged solves (Burgers, CFL 0.5)
  reaches the same tolerance in fewer CG iterations inside the time steps,
  and the state agrees with the plain form's to the solver tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S     # noqa: E402
from tests.helpers import oracle_ml, oracle_space, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def _case(name):
    if name == "burgers":
        w = inputs.scaled("burgers2d", nel=(5, 5))
        X, Y = oracle_space(w, w["levels"][-1]).coords()
        u0 = inputs.burgers2d_initial(X, Y)
    else:
        w = dict(inputs.scaled("ns_shear", nel=(6, 5)), Re=200.0)
        X, Y = oracle_space(w, w["levels"][-1]).coords()
        u0 = inputs.shear_layer(X, Y, w["gamma"], w["mach"], delta=0.08)
    P = w["levels"][-1]["P"]
    dt = inputs.cfl_dt(0.5, 1.0 / w["levels"][-1]["nel"][0], P, inputs.max_wave_speed(w["pde"], u0))
    return w, u0, dt


@pytest.mark.parametrize("name", ["burgers", "ns"])
def test_learned_sweep_step_parity(dev, name):
    w, u0, dt = _case(name)
    ctx = S.Context(w, cg_rtol=1e-14, cg_maxit=10000)
    fine = len(w["levels"]) - 1
    m = S.sisdc_mlp_create(ctx.levels[fine], 32, seed=9, bf16=1)
    S.sisdc_set_learned(ctx.ctx, fine, m)
    om = oracle_ml(w)
    u = u0.copy()
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    worst = 0.0
    for n in range(2):
        u = om.step(u, dt, 2, start="cascade")
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 2, S.SISDC_START_CASCADE, 1)
        worst = max(worst, rel_l2(du.cpu().numpy(), u))
    S.sisdc_sync(ctx.ctx)
    S.sisdc_set_learned(ctx.ctx, fine, None)
    S.sisdc_mlp_destroy(m)
    ctx.close()
    assert worst < 1e-12


def test_learned_sweep_saves_iterations_inside_steps(dev):
    w = inputs.scaled("burgers2d", nel=(8, 8))
    X, Y = oracle_space(w, w["levels"][-1]).coords()
    u0 = inputs.burgers2d_initial(X, Y)
    dt = inputs.cfl_dt(0.5, 1.0 / 8, 7, inputs.max_wave_speed("burgers", u0))
    fine = 1
    # training data: the plain method's own fine-level solves
    ctx = S.Context(w, cg_rtol=1e-10, cg_maxit=2000)
    nc, n, M = ctx.info(fine)
    cap = 400
    lr_ = torch.zeros((cap, nc * n), dtype=torch.float64, device=dev)
    ldx = torch.zeros_like(lr_)
    lc = torch.zeros(cap, dtype=torch.float64, device=dev)
    S.sisdc_set_solve_log(ctx.ctx, fine, lr_, ldx, lc, cap)
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    for k in range(12):
        S.sisdc_step(ctx.ctx, du, k * dt, dt, 3, S.SISDC_START_CASCADE, 1)
    S.sisdc_sync(ctx.ctx)
    nlog = S.sisdc_get_solve_log_count(ctx.ctx)
    cs = lc[:nlog].cpu().numpy()
    keep = np.nonzero(torch.abs(ldx[:nlog]).amax(dim=1).cpu().numpy() > 0)[0]
    m = S.sisdc_mlp_create(ctx.levels[fine], 64, seed=3, bf16=1)
    S.sisdc_mlp_train(m, lr_[keep].contiguous(), ldx[keep].contiguous(), cs[keep], len(keep), 60, 1e-3)
    S.sisdc_set_solve_log(ctx.ctx, fine)
    ctx.close()
    # the next steps (not trained on) with and without the learned guess
    start = du.clone()
    res = {}
    for learned in (False, True):
        c2 = S.Context(w, cg_rtol=1e-10, cg_maxit=2000)
        if learned:
            S.sisdc_set_learned(c2.ctx, fine, m)
        u = start.clone()
        S.sisdc_reset_stats(c2.ctx)
        for k in range(4):
            S.sisdc_step(c2.ctx, u, (12 + k) * dt, dt, 3, S.SISDC_START_CASCADE, 1)
        S.sisdc_sync(c2.ctx)
        st = S.sisdc_get_stats(c2.ctx)
        res[learned] = (st["cg_iters"], st["cg_solves"], u.clone())
        if learned:
            S.sisdc_set_learned(c2.ctx, fine, None)
        c2.close()
    S.sisdc_mlp_destroy(m)
    (ip, sp_, up), (il, sl, ul) = res[False], res[True]
    print("burgers 8x8 CFL 0.5, 4 steps: plain %d CG iterations in %d solves, learned guess %d in %d"
          % (ip, sp_, il, sl))
    assert sl == sp_
    assert il < ip
    assert float(torch.linalg.vector_norm(ul - up) / torch.linalg.vector_norm(up)) < 1e-7
