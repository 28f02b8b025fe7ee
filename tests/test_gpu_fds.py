"""The element-wise fast-diagonalisation preconditioner (sisdc_solve_fds)
against the oracle's FDS-PCG, and its cost against Jacobi-PCG.

* parity: the same system solved by the CUDA kernel and by the oracle with
  the same preconditioner and stopping rule (rtol 1e-14): solutions within
  1e-12 (relative L2), iteration counts within one;
* comparison on the fine level of the 2D Burgers workload (32 x 32
  elements, P = 7, two components) at CFL 0.5, 4 and 32: iterations and
  CUDA-event time per solve for Jacobi and FDS, from the same warm start
  (the previous time level), both to rtol 1e-12 -- printed for the record;
  both reach the same solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.fds import pcg_fds                             # noqa: E402
from paper_2504_18526_gb300 import inputs, sisdc as S     # noqa: E402
from tests.helpers import oracle_space, rel_l2             # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


CASES = [
    dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=0.01, lo=(0.0, 0.0), hi=(2.0, 0.0),
         nodes="radau_right", levels=[dict(nel=(9, 1), P=6, M=3)]),
    dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=0.01, lo=(0.0, 0.0), hi=(2.0, 0.0),
         nodes="radau_right", levels=[dict(nel=(5, 1), P=15, M=3)]),
    dict(pde="convdiff", dim=2, ncomp=1, adv=(1.0, 0.5), nu=0.01, lo=(0.0, 0.0), hi=(1.0, 2.0),
         nodes="radau_right", levels=[dict(nel=(5, 3), P=3, M=3)]),
    dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
         levels=[dict(nel=(4, 6), P=7, M=3)]),
    dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
         levels=[dict(nel=(3, 3), P=8, M=3)]),
]


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("c", [1e-4, 3e-2])
def test_fds_solve_parity(dev, k, c):
    w = CASES[k]
    lvd = w["levels"][0]
    sp = oracle_space(w, lvd, rtol=1e-14)
    rng = np.random.default_rng(100 + k)
    rhs = rng.standard_normal(sp.shape)
    x0 = rng.standard_normal(sp.shape)
    want, it_ref = pcg_fds(sp, c, rhs, x0, 1e-14, 10000)
    ctx = S.Context(w, cg_rtol=1e-14, cg_maxit=10000)
    x = torch.from_numpy(x0.ravel().copy()).to(dev)
    it = S.sisdc_solve_fds(ctx.levels[0], c, torch.from_numpy(rhs.ravel().copy()).to(dev), x, want_iters=True)
    S.sisdc_sync(ctx.ctx)
    ctx.close()
    assert rel_l2(x.cpu().numpy(), want) <= 1e-12
    assert abs(it - it_ref) <= 1, (it, it_ref)


def test_fds_against_jacobi_on_burgers_level(dev):
    w = inputs.scaled("burgers2d", levels=[dict(nel=(32, 32), P=7, M=5)])
    ctx = S.Context(w, cg_rtol=1e-12, cg_maxit=5000)
    lv = ctx.levels[0]
    nc, n, M = ctx.info(0)
    hx, hy = np.zeros(n), np.zeros(n)
    S.sisdc_level_coords(lv, hx, hy)
    u0 = inputs.initial_state("burgers2d", hx, hy)
    lam = inputs.max_wave_speed("burgers", u0)
    ut = torch.from_numpy(np.ascontiguousarray(u0).ravel()).to(dev)
    # a right-hand side one substep ahead: the state advected by a forward
    # Euler step of the smooth initial field (any smooth field would do)
    rhs = ut * (1.0 - 0.01) + 0.01 * torch.roll(ut, 1)
    rows = []
    for cfl in (0.5, 4.0, 32.0):
        dt = inputs.cfl_dt(cfl, 1.0 / 32, 7, lam)
        dtm = 0.28 * dt
        c = dtm * (w["nu"] + 0.5 * dtm * lam * lam)
        res = {}
        for name, fn in (("jacobi", S.sisdc_solve), ("fds", S.sisdc_solve_fds)):
            x = ut.clone()
            it = fn(lv, c, rhs, x, want_iters=True)  # iterations (and warm-up)
            x = ut.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn(lv, c, rhs, x)
            e1.record()
            torch.cuda.synchronize()
            res[name] = (it, e0.elapsed_time(e1), x)
        S.sisdc_sync(ctx.ctx)
        rel = float(torch.linalg.vector_norm(res["fds"][2] - res["jacobi"][2]) / torch.linalg.vector_norm(res["jacobi"][2]))
        assert rel < 1e-9
        rows.append("CFL %5.1f c=%.3e: Jacobi %3d it %.3f ms | FDS %3d it %.3f ms" % (
            cfl, c, res["jacobi"][0], res["jacobi"][1], res["fds"][0], res["fds"][1]))
    ctx.close()
    print("burgers2d fine level (32^2, P=7, 2 comps), warm start from the old state:\n  " + "\n  ".join(rows))
