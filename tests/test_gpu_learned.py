"""The learned initial guess / preconditioner of the implicit stage.

* forward/backward parity of the CUDA training kernels against the FP64
  oracle MLP (FP32 mode: 1e-5; BF16 tensor-core mode: 2e-3 against the
  oracle with every GEMM operand rounded to bfloat16);
* training on (initial residual, correction) pairs logged from the method's
  own implicit solves lowers the loss;
* on held-out logged solves, the learned initial guess reaches the same
  tolerance in fewer CG iterations than plain Jacobi-PCG (the element-wise
  fast-diagonalisation preconditioner is counted beside it).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp                             # noqa: E402
from paper_2504_18526_gb300 import inputs, sisdc as S     # noqa: E402
from tests.helpers import oracle_space                     # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def unpack(theta, n_in, H, q):
    o = 0
    p = {}
    for name, shape in (("W1", (n_in, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (H, q)), ("b3", (q,))):
        n = int(np.prod(shape))
        p[name] = theta[o:o + n].reshape(shape).astype(np.float64)
        o += n
    return p


def pack(g):
    return np.concatenate([g[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("use_bf16", [0, 1])
def test_mlp_loss_and_gradient_parity(dev, use_bf16):
    w = dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
             levels=[dict(nel=(5, 4), P=3, M=3)])
    ctx = S.Context(w)
    m = S.sisdc_mlp_create(ctx.levels[0], 24, seed=7, bf16=use_bf16)
    n_in, H, q, npar = S.sisdc_mlp_info(m)
    sp = oracle_space(w, w["levels"][0])
    rng = np.random.default_rng(11)
    r = rng.standard_normal(sp.shape)
    dx = 0.1 * rng.standard_normal(sp.shape)
    c = 3e-3
    theta = np.zeros(npar, dtype=np.float32)
    S.sisdc_mlp_params(m, get=theta)
    grad = np.zeros(npar, dtype=np.float32)
    loss = S.sisdc_mlp_loss_grad(m, torch.from_numpy(r).to(dev), torch.from_numpy(dx).to(dev), c, grad)
    p = unpack(theta, n_in, H, q)
    if use_bf16:
        for k in ("W1", "W2", "W3"):
            p[k] = bf16(p[k])
    X, s = omlp.patches(r, sp.nex, sp.ney, q, c, min(sp.hx, sp.hy))
    T = omlp.targets(r, dx, s, q)
    # BF16 mode: the tensor-core GEMMs round both operands of every product
    # to bfloat16, which the oracle reproduces with round_op
    rnd = omlp.bf16_round if use_bf16 else None
    l_ref, g_ref = omlp.loss_and_grads(p, X, T, round_op=rnd)
    tol = 2e-3 if use_bf16 else 1e-5
    assert abs(loss - l_ref) <= tol * abs(l_ref)
    gr = pack(g_ref)
    assert np.linalg.norm(grad - gr) <= tol * np.linalg.norm(gr)
    # inference: z = r + s * MLP(patch / s)
    z = torch.zeros(sp.shape, dtype=torch.float64, device=dev)
    S.sisdc_mlp_apply(m, torch.from_numpy(r).to(dev), c, z)
    zr = omlp.apply(p, r, sp.nex, sp.ney, q, c, min(sp.hx, sp.hy), round_op=rnd)
    torch.cuda.synchronize()
    assert np.linalg.norm(z.cpu().numpy() - zr) <= tol * np.linalg.norm(zr)
    S.sisdc_mlp_destroy(m)
    ctx.close()


def _workload(name):
    """A small case of a workload at the workloads' own CFL number 0.5, where
    the implicit solves need tens of CG iterations: (workload, initial
    state, dt)."""
    if name == "burgers":
        w = inputs.scaled("burgers2d", nel=(8, 8))
        X, Y = oracle_space(w, w["levels"][-1]).coords()
        u0 = inputs.burgers2d_initial(X, Y)
    else:   # Navier-Stokes shear layer, smoothed to the coarse grid, Re = 200
        w = dict(inputs.scaled("ns_shear", nel=(8, 8)), Re=200.0)
        X, Y = oracle_space(w, w["levels"][-1]).coords()
        u0 = inputs.shear_layer(X, Y, w["gamma"], w["mach"], delta=0.06)
    P = w["levels"][-1]["P"]
    return w, u0, inputs.cfl_dt(0.5, 1.0 / 8, P, inputs.max_wave_speed(w["pde"], u0))


@pytest.mark.parametrize("name", ["burgers", "ns"])
def test_learned_initial_guess_saves_iterations(dev, name):
    w, u0, dt = _workload(name)
    ctx = S.Context(w, cg_rtol=1e-10, cg_maxit=2000)
    fine = len(w["levels"]) - 1
    nc, n, M = ctx.info(fine)
    cap = 160
    lr_ = torch.zeros((cap, nc * n), dtype=torch.float64, device=dev)
    ldx = torch.zeros_like(lr_)
    lc = torch.zeros(cap, dtype=torch.float64, device=dev)
    S.sisdc_set_solve_log(ctx.ctx, fine, lr_, ldx, lc, cap)
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    for k in range(6):
        S.sisdc_step(ctx.ctx, du, k * dt, dt, 3, S.SISDC_START_CASCADE, 1)
    S.sisdc_sync(ctx.ctx)
    nlog = S.sisdc_get_solve_log_count(ctx.ctx)
    assert nlog >= 100
    cs = lc[:nlog].cpu().numpy()
    keep = np.nonzero(torch.abs(ldx[:nlog]).amax(dim=1).cpu().numpy() > 0)[0]
    train, test = keep[: int(0.8 * len(keep))], keep[int(0.8 * len(keep)):]
    lv = ctx.levels[fine]
    m = S.sisdc_mlp_create(lv, 64, seed=3, bf16=1)
    def mean_loss(idx):
        return np.mean([S.sisdc_mlp_loss_grad(m, lr_[k], ldx[k], float(cs[k])) for k in idx])

    l0_tr, l0_te = mean_loss(train), mean_loss(test)
    rtr, dtr = lr_[train].contiguous(), ldx[train].contiguous()
    S.sisdc_mlp_train(m, rtr, dtr, cs[train], len(train), 120, 1e-3)
    l1_tr, l1_te = mean_loss(train), mean_loss(test)
    print("loss train %.3e -> %.3e, held-out %.3e -> %.3e" % (l0_tr, l1_tr, l0_te, l1_te))
    assert l1_tr < 0.5 * l0_tr and l1_te < 0.5 * l0_te
    plain = learned = flexible = fds = 0
    for k in test:
        rhs = lr_[k].contiguous()                 # (I - cL) x = r0 (nodal), x* = logged correction
        x = torch.zeros_like(rhs)
        plain += S.sisdc_solve_learned(lv, m, float(cs[k]), rhs, x, 0)
        x2 = torch.zeros_like(rhs)
        learned += S.sisdc_solve_learned(lv, m, float(cs[k]), rhs, x2, 1)
        torch.cuda.synchronize()
        # both meet the same tolerance on the same system: the solutions agree
        assert float(torch.linalg.vector_norm(x2 - x) / torch.linalg.vector_norm(x)) < 1e-8
        x3 = torch.zeros_like(rhs)
        flexible += S.sisdc_solve_learned(lv, m, float(cs[k]), rhs, x3, 2)
        torch.cuda.synchronize()
        assert float(torch.linalg.vector_norm(x3 - x) / torch.linalg.vector_norm(x)) < 1e-8
        x4 = torch.zeros_like(rhs)                # the non-learned separable preconditioner
        fds += S.sisdc_solve_fds(lv, float(cs[k]), rhs, x4, want_iters=True)
        torch.cuda.synchronize()
        assert float(torch.linalg.vector_norm(x4 - x) / torch.linalg.vector_norm(x)) < 1e-8
    S.sisdc_sync(ctx.ctx)
    print("%s held-out solves %d: plain PCG %d iterations, learned guess + PCG %d, learned flexible CG %d, "
          "element-wise FDS-PCG %d" % (name, len(test), plain, learned, flexible, fds))
    assert learned < plain
    S.sisdc_mlp_destroy(m)
    S.sisdc_set_solve_log(ctx.ctx, fine)
    ctx.close()
