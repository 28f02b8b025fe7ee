"""2:1 h-coarsening between levels (Sec. 6.2) through the C ABI against the
CPU oracle: the four space-time transfers element by element (1e-14), and
whole time steps of h-coarsened multilevel methods (1e-12): the paper's
1D convection-diffusion level structure (elements doubling from level to
level at equal degree; here 4/8/16 elements of degree 6 with M = 3/5/7
Radau-Right nodes) and 2D Burgers with h- and p-coarsening in one step,
both solution projections."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.mlsdc import Transfer                          # noqa: E402
from paper_2504_18526_gb300 import inputs, sisdc as S     # noqa: E402
from tests.helpers import oracle_ml, oracle_space, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


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


CD1D = dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=1e-3, lo=(0.0, 0.0), hi=(1.0, 0.0),
            nodes="radau_right",
            levels=[dict(nel=(4, 1), P=6, M=3), dict(nel=(8, 1), P=6, M=5), dict(nel=(16, 1), P=6, M=7)])
BURG = dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
            levels=[dict(nel=(3, 2), P=3, M=3), dict(nel=(6, 4), P=5, M=5)])
MIXED = dict(pde="convdiff", dim=2, ncomp=1, adv=(0.8, -0.6), nu=0.01, lo=(0.0, 0.0), hi=(1.0, 2.0),
             nodes="lobatto",
             levels=[dict(nel=(3, 4), P=4, M=3), dict(nel=(6, 4), P=4, M=5)])
CASES = {"cd1d": CD1D, "burgers": BURG, "mixed_ratio": MIXED}


@pytest.mark.parametrize("projection", ["interp", "l2"])
@pytest.mark.parametrize("case", list(CASES))
def test_h_transfer_parity(dev, case, projection):
    w = CASES[case]
    ctx = S.Context(w, cg_rtol=1e-14, cg_maxit=10000, projection=projection)
    om = oracle_ml(w, projection=projection)
    for l in range(1, len(om.levels)):
        Tr = Transfer(om.levels[l], om.levels[l - 1], projection)
        fs, cs = om.levels[l].space, om.levels[l - 1].space
        Mf, Mc = om.levels[l].M, om.levels[l - 1].M
        rng = np.random.default_rng(10 + l)
        Uf = rng.standard_normal((Mf,) + fs.shape)
        Uc = rng.standard_normal((Mc,) + cs.shape)
        fine, coarse = ctx.levels[l], ctx.levels[l - 1]
        out_f = torch.empty((Mf,) + fs.shape, dtype=torch.float64, device=dev)
        out_c = torch.empty((Mc,) + cs.shape, dtype=torch.float64, device=dev)
        S.sisdc_transfer(fine, coarse, S.T_INTERP, T(Uc, dev), out_f)
        assert rel_l2(N(out_f), Tr.interp(Uc)) < 1e-14
        S.sisdc_transfer(fine, coarse, S.T_PROJECT, T(Uf, dev), out_c)
        assert rel_l2(N(out_c), Tr.project(Uf)) < 1e-14
        S.sisdc_transfer(fine, coarse, S.T_RESTRICT, T(Uf, dev), out_c)
        assert rel_l2(N(out_c), Tr.restrict(Uf)) < 1e-14
        oc = torch.empty(cs.shape, dtype=torch.float64, device=dev)
        S.sisdc_transfer(fine, coarse, S.T_PROJECT_SPACE, T(Uf[0], dev), oc)
        assert rel_l2(N(oc), Tr.project_space(Uf[0])) < 1e-14
    S.sisdc_sync(ctx.ctx)
    ctx.close()


@pytest.mark.parametrize("case,start,projection", [("cd1d", "fmg1", "interp"), ("cd1d", "predictor", "l2"),
                                                   ("burgers", "cascade", "interp"),
                                                   ("mixed_ratio", "cascade", "l2")])
def test_h_coarsened_step_parity(dev, case, start, projection):
    w = CASES[case]
    sp = oracle_space(w, w["levels"][-1])
    X, Y = sp.coords()
    if case == "cd1d":
        u0 = (np.sin(2 * math.pi * X) + 0.5 * np.cos(6 * math.pi * X))[None]
        dt = 0.02
    elif case == "burgers":
        u0 = inputs.burgers2d_initial(X, Y)
        dt = inputs.cfl_dt(0.5, 1.0 / 6, 5, inputs.max_wave_speed("burgers", u0))
    else:
        u0 = (np.sin(2 * math.pi * X) * np.cos(math.pi * Y))[None]
        dt = 0.01
    ctx = S.Context(w, cg_rtol=1e-14, cg_maxit=10000, projection=projection)
    om = oracle_ml(w, projection=projection)
    u = u0.copy()
    du = T(u0, dev)
    worst = 0.0
    for n in range(3):
        u = om.step(u, dt, 2, start=start)
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 2, S.START_IDS[start], 1)
        worst = max(worst, rel_l2(N(du), u))
    S.sisdc_sync(ctx.ctx)
    ctx.close()
    assert worst < 1e-12 and np.max(np.abs(u - u0)) > 1e-6
