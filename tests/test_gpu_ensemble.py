"""Batched ensemble of independent 2D convection-diffusion problems: every
instance of one CUDA ensemble step must equal the same instance stepped
alone, by the CPU oracle (relative L2 <= 1e-12, FP64) and by the
single-problem CUDA path, whatever the tile shapes; the mixed-precision form
stays within 1.05x of the FP64 form's error against the exact solution."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S     # noqa: E402
from oracle.dg import ConvDiff, DGSpace                    # noqa: E402
from oracle.mlsdc import MLSDC                             # noqa: E402
from oracle.sdc import Level                               # noqa: E402
from tests.helpers import rel_l2                           # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def space(inst, P, rtol=1e-14):
    return DGSpace(2, tuple(inst["nel"]), P, (0.0, 0.0), (1.0, 1.0), ConvDiff(inst["adv"], inst["nu"]),
                   cg_rtol=rtol, cg_maxit=10000)


def initial(inst):
    X, Y = space(inst, inst["P"]).coords()
    return inputs.ensemble_exact(inst, X, Y, 0.0)[0]


def oracle_steps(inst, nsteps, M=5, Mc=3, nodes="radau_right", stages=2, ncycles=3, start="cascade"):
    P = inst["P"]
    levels = [Level(space(inst, (P + 1) // 2), nodes, Mc), Level(space(inst, P), nodes, M)]
    ml = MLSDC(levels, stages=stages, Nc=2)
    u = initial(inst)[None]
    for _ in range(nsteps):
        u = ml.step(u, inst["dt"], ncycles, start=start, post_sweep=True)
    return u[0]


def pack(E, dev):
    u = np.zeros(E.total)
    for k, d in enumerate(E.instances):
        u[E.offsets[k]:E.offsets[k] + E.size(k)] = initial(d).ravel()
    return torch.from_numpy(u).to(dev)


def unpack(E, u, k):
    torch.cuda.synchronize()
    return u[E.offsets[k]:E.offsets[k] + E.size(k)].cpu().numpy()


def small_instances():
    """One instance per degree 2..8 on small uneven grids, random nu, a, dt."""
    rng = np.random.default_rng(20250418)
    grids = [(2, 3), (3, 2), (3, 3), (4, 2), (2, 4), (3, 4), (4, 3)]
    out = []
    for k, P in enumerate(range(2, 9)):
        th = rng.uniform(0, 2 * math.pi)
        ne = grids[k]
        out.append(dict(nel=ne, P=P, nu=float(10 ** rng.uniform(-3, -1.5)), adv=(math.cos(th), math.sin(th)),
                        dt=inputs.cfl_dt(0.5, 1.0 / max(ne), P, 1.0) * rng.uniform(1.0, 4.0),
                        seed=100 + k))
    # a second instance of degree 5 so that one group holds several instances
    out.append(dict(nel=(5, 3), P=5, nu=2e-3, adv=(0.6, -0.8), dt=4e-3, seed=200))
    return out


@pytest.mark.parametrize("variant", ["radau_si2_cascade", "lobatto_si1_predictor"])
@pytest.mark.parametrize("tiles", ["default", "ragged"])
def test_ensemble_matches_oracle_per_instance(dev, variant, tiles):
    insts = small_instances()
    kw = (dict(nodes="radau_right", si_stages=2, start="cascade") if variant == "radau_si2_cascade"
          else dict(nodes="lobatto", si_stages=1, start="predictor"))
    E = S.Ensemble(insts, cg_rtol=1e-14, cg_maxit=500, use_graph=0, **kw)
    if tiles == "ragged":
        # several tiles per instance with a ragged last tile, few blocks:
        # blocks own tiles of several instances and instances span blocks
        for g in range(S.sisdc_ens_num_groups(E.ens)):
            S.sisdc_ens_set_tiles(E.ens, g, 1, 2, 3)
            S.sisdc_ens_set_tiles(E.ens, g, 0, 4, 2)
    u = pack(E, dev)
    S.sisdc_ens_step(E.ens, u, 2)
    S.sisdc_ens_sync(E.ens)
    for k, d in enumerate(insts):
        ref = oracle_steps(d, 2, nodes=kw["nodes"], stages=kw["si_stages"], start=kw["start"])
        got = unpack(E, u, k).reshape(ref.shape)
        assert rel_l2(got, ref) <= TOL, (k, d["P"], rel_l2(got, ref))
    st = S.sisdc_ens_get_stats(E.ens, len(insts))
    assert st["cg_noconv"] == 0 and st["cg_solves"] > 0
    assert np.all(st["inst_iters"] > 0)
    E.close()


def single_path_steps(d, u0, nsteps, dev, precision=S.SISDC_FP64, rtol=1e-14):
    w = dict(pde="convdiff", dim=2, ncomp=1, adv=d["adv"], nu=d["nu"], lo=(0.0, 0.0), hi=(1.0, 1.0),
             nodes="radau_right",
             levels=[dict(nel=d["nel"], P=(d["P"] + 1) // 2, M=3), dict(nel=d["nel"], P=d["P"], M=5)])
    ctx = S.Context(w, cg_rtol=rtol, cg_maxit=500, precision=precision)
    u = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    for _ in range(nsteps):
        S.sisdc_step(ctx.ctx, u, 0.0, d["dt"], 3, S.SISDC_START_CASCADE, 1)
    S.sisdc_sync(ctx.ctx)
    out = u.cpu().numpy()
    ctx.close()
    return out


def test_ensemble_matches_single_problem_path_and_autotune(dev):
    """Workload-shaped instances (a sample of the 512-instance draw, grids
    capped for time): ensemble (graph-captured) == single-problem CUDA path,
    before and after the autotuner changes the tile shapes."""
    insts = inputs.ensemble_instances(24)
    insts = [dict(d, nel=(min(d["nel"][0], 16), min(d["nel"][1], 16))) for d in insts]
    E = S.Ensemble(insts, cg_rtol=1e-14, cg_maxit=500, use_graph=1)
    u0 = pack(E, dev)
    refs = [single_path_steps(d, initial(d).ravel(), 2, dev) for d in insts]
    for tuned in (False, True):
        if tuned:
            cfg = S.sisdc_ens_autotune(E.ens, u0, 1)
            assert cfg.shape == (2 * S.sisdc_ens_num_groups(E.ens), 4)
            assert np.all(cfg[:, 2] >= 1) and np.all(cfg[:, 3] >= 1)
        u = u0.clone()
        S.sisdc_ens_step(E.ens, u, 2)
        S.sisdc_ens_sync(E.ens)
        for k, d in enumerate(insts):
            assert rel_l2(unpack(E, u, k), refs[k]) <= TOL, (tuned, k)
    E.close()


@pytest.mark.parametrize("precision", [S.SISDC_FP64, S.SISDC_MIXED])
def test_register_capped_kernel(dev, precision):
    """A grid of two blocks per SM with the largest tiles runs the
    register-capped kernel (at most 64 registers per thread): the same
    results as one block per SM (the plain kernel) up to the order of the
    per-instance partial sums, which follows the grid."""
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    insts = [dict(nel=(131, 131), P=3, nu=3e-3, adv=(0.6, 0.8), dt=1e-3, seed=11),
             dict(nel=(78, 78), P=8, nu=1e-3, adv=(-0.8, 0.6), dt=5e-4, seed=12)]
    out = []
    for blocks in (1, 2):
        E = S.Ensemble(insts, cg_rtol=1e-12, cg_maxit=500, use_graph=1, precision=precision)
        for g in range(S.sisdc_ens_num_groups(E.ens)):
            for fine in (0, 1):
                P = int(S.sisdc_ens_config(E.ens)[2 * g + (0 if fine else 1)][1])
                S.sisdc_ens_set_tiles(E.ens, g, fine, max(1, 512 // ((P + 1) ** 2)), blocks * nsm)
        cfg = S.sisdc_ens_config(E.ens)
        assert np.all(cfg[:, 3] == blocks * nsm)        # every level has enough tiles
        u = pack(E, dev)
        S.sisdc_ens_step(E.ens, u, 2)
        S.sisdc_ens_sync(E.ens)
        out.append(u.cpu().numpy())
        st = S.sisdc_ens_get_stats(E.ens, len(insts))
        assert st["cg_noconv"] == 0 and st["cg_solves"] > 0
        E.close()
    assert rel_l2(out[1], out[0]) <= (TOL if precision == S.SISDC_FP64 else 1e-9)


def exact_error(d, u, t):
    """Continuous L2 error (GLL quadrature) against the exact solution."""
    sp = space(d, d["P"])
    X, Y = sp.coords()
    ex = inputs.ensemble_exact(d, X, Y, t)
    return sp.l2(u.reshape(ex.shape) - ex)


def test_mixed_precision_error_within_bar(dev):
    """FP32 inner CG + FP64 refinement: per instance, the error against the
    exact solution after 10 steps is at most 1.05x the FP64 form's."""
    insts = inputs.ensemble_instances(12)
    insts = [dict(d, nel=(min(d["nel"][0], 12), min(d["nel"][1], 12))) for d in insts]
    res, irs = {}, {}
    # FP64; mixed on both levels; mixed on the fine level only (mixed_levels bit 1)
    for key, prec, ml in (("fp64", S.SISDC_FP64, 0), ("mixed", S.SISDC_MIXED, 0), ("fine", S.SISDC_MIXED, 2)):
        E = S.Ensemble(insts, cg_rtol=1e-12, cg_maxit=500, use_graph=1, precision=prec, mixed_levels=ml)
        u = pack(E, dev)
        S.sisdc_ens_step(E.ens, u, 10)
        S.sisdc_ens_sync(E.ens)
        res[key] = [unpack(E, u, k) for k in range(len(insts))]
        irs[key] = S.sisdc_ens_get_stats(E.ens)["ir_steps"]
        E.close()
    assert irs["fp64"] == 0 and 0 < irs["fine"] < irs["mixed"]
    for k, d in enumerate(insts):
        e64 = exact_error(d, res["fp64"][k], 10 * d["dt"])
        for key in ("mixed", "fine"):
            emx = exact_error(d, res[key][k], 10 * d["dt"])
            assert emx <= 1.05 * e64 + 1e-14, (key, k, e64, emx)


def test_full_ensemble_sampled_parity(dev):
    """The 512-instance workload at full size, one graph-captured step: the
    smallest instances against the oracle, the largest against the
    single-problem CUDA path (both relative L2 <= 1e-12)."""
    insts = inputs.ensemble_instances()
    E = S.Ensemble(insts, cg_rtol=1e-14, cg_maxit=500, use_graph=1)
    u = pack(E, dev)
    S.sisdc_ens_step(E.ens, u, 1)
    S.sisdc_ens_sync(E.ens)
    size = [E.size(k) for k in range(len(insts))]
    order = np.argsort(size)
    for k in order[:4]:
        ref = oracle_steps(insts[k], 1)
        assert rel_l2(unpack(E, u, k).reshape(ref.shape), ref) <= TOL, k
    for k in order[-2:]:
        ref = single_path_steps(insts[k], initial(insts[k]).ravel(), 1, dev)
        assert rel_l2(unpack(E, u, k), ref) <= TOL, k
    st = S.sisdc_ens_get_stats(E.ens, len(insts))
    assert st["cg_noconv"] == 0 and np.all(st["inst_iters"] > 0)
    E.close()
