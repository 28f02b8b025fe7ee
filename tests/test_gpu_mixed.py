"""Mixed-precision form (FP32 operators and inner CG; FP64 state, S.F
quadrature, right-hand sides, inner products and refinement residual).

The bar: its error against a reference solution is never worse than 1.05x
the error of the plain FP64 form.  References: the exact translated vortex
(Euler) and, for Burgers, an FP64 oracle run at dt/4 with enough V-cycles to
reach the collocation solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S   # noqa: E402
from tests.helpers import oracle_ml, oracle_space, rel_l2   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def run(w, u0, dt, nsteps, ncycles, start, dev, precision, rtol=1e-12, mixed_levels=0):
    ctx = S.Context(w, precision=precision, cg_rtol=rtol, cg_maxit=2000, mixed_levels=mixed_levels)
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    for n in range(nsteps):
        S.sisdc_step(ctx.ctx, du, n * dt, dt, ncycles, S.START_IDS[start], 1)
    S.sisdc_sync(ctx.ctx)
    st = S.sisdc_get_stats(ctx.ctx)
    ctx.close()
    torch.cuda.synchronize()
    return du.cpu().numpy(), st


def test_mixed_close_to_fp64(dev):
    w = inputs.scaled("burgers2d", nel=(6, 6))
    X, Y = oracle_space(w, w["levels"][-1]).coords()
    u0 = inputs.burgers2d_initial(X, Y)
    dt = inputs.cfl_dt(0.5, 1.0 / 6, 7, inputs.max_wave_speed("burgers", u0))
    u64, _ = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_FP64)
    u32, st = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_MIXED)
    assert rel_l2(u32, u64) < 1e-6
    assert st["ir_steps"] > 0 and st["cg_noconv"] == 0


def test_mixed_levels_selects_levels(dev):
    """mixed_levels selects the levels that run the mixed form: refinement
    steps appear only for the selected level (fewer than with every level
    mixed), each selection gives a different result from the all-FP64 and
    all-mixed runs, and every result stays within the mixed form's distance
    of the FP64 one."""
    w = inputs.scaled("burgers2d", nel=(6, 6))
    X, Y = oracle_space(w, w["levels"][-1]).coords()
    u0 = inputs.burgers2d_initial(X, Y)
    dt = inputs.cfl_dt(0.5, 1.0 / 6, 7, inputs.max_wave_speed("burgers", u0))
    nl = len(w["levels"])
    u64, s64 = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_FP64)
    uall, sall = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_MIXED)
    ufin, sfin = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_MIXED, mixed_levels=1 << (nl - 1))
    ucrs, scrs = run(w, u0, dt, 3, 3, "cascade", dev, S.SISDC_MIXED, mixed_levels=1)
    assert s64["ir_steps"] == 0
    assert 0 < sfin["ir_steps"] < sall["ir_steps"] and 0 < scrs["ir_steps"] < sall["ir_steps"]
    for u in (uall, ufin, ucrs):
        assert rel_l2(u, u64) < 1e-6
    assert not np.array_equal(ufin, u64) and not np.array_equal(ufin, uall)


def test_mixed_levels_rejects_unsupported_level(dev):
    """The mixed form needs P >= 3; a P = 2 level that is not selected is fine."""
    w = inputs.scaled("burgers2d", nel=(4, 4))
    w = dict(w, levels=[dict(w["levels"][0], P=2), w["levels"][-1]])
    with pytest.raises(Exception):
        S.Context(w, precision=S.SISDC_MIXED)
    ctx = S.Context(w, precision=S.SISDC_MIXED, mixed_levels=2)
    ctx.close()


def test_mixed_equal_error_burgers(dev):
    """Tuned vs plain at equal L2 error on Burgers (reference: FP64 oracle at
    dt/4, 6 V-cycles per step)."""
    w = inputs.scaled("burgers2d", nel=(8, 8))
    sp = oracle_space(w, w["levels"][-1])
    X, Y = sp.coords()
    u0 = inputs.burgers2d_initial(X, Y)
    dt = inputs.cfl_dt(0.5, 1.0 / 8, 7, inputs.max_wave_speed("burgers", u0))
    nsteps = 12
    om = oracle_ml(w, rtol=1e-13)
    uref = u0.copy()
    for _ in range(4 * nsteps):
        uref = om.step(uref, dt / 4, 6)
    up, _ = run(w, u0, dt, nsteps, 3, "cascade", dev, S.SISDC_FP64)
    ut, _ = run(w, u0, dt, nsteps, 3, "cascade", dev, S.SISDC_MIXED)
    ep, et = sp.l2(up - uref), sp.l2(ut - uref)
    print("burgers: plain error %.4e, mixed error %.4e" % (ep, et))
    assert ep > 0 and et <= 1.05 * ep


def test_mixed_equal_error_euler_vortex(dev):
    """Tuned vs plain at equal L2 error against the exact translated vortex."""
    w = inputs.scaled("euler_vortex", nel=(8, 8))
    sp = oracle_space(w, w["levels"][-1])
    X, Y = sp.coords()
    u0 = inputs.isentropic_vortex(X, Y)
    dt = inputs.cfl_dt(0.5, 20.0 / 8, 7, inputs.max_wave_speed("euler", u0))
    nsteps = 10
    up, _ = run(w, u0, dt, nsteps, 3, "fmg1", dev, S.SISDC_FP64)
    ut, _ = run(w, u0, dt, nsteps, 3, "fmg1", dev, S.SISDC_MIXED)
    ue = inputs.isentropic_vortex(X, Y, nsteps * dt)
    ep, et = sp.l2(up - ue), sp.l2(ut - ue)
    print("euler: plain error %.4e, mixed error %.4e" % (ep, et))
    assert et <= 1.05 * ep
