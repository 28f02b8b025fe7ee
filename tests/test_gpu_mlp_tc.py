"""The fused tcgen05 forward pass of the element-patch MLP (sisdc_mlp_apply,
BF16 mode) against the warp-level mma.sync path and against the FP64 oracle
MLP with every GEMM operand rounded to bfloat16 (the same operands: the
patch rows, weights and hidden activations in BF16, FP32 accumulation).

Cases: the Navier-Stokes level shape (P = 5, four components, 325 inputs,
hidden width 112, 36 outputs) and a Burgers level (P = 7, two components,
577 inputs: ten 64-wide K panels, hidden width 64), with the row count not
a multiple of the 128-row tile; overwrite and accumulate modes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp                             # noqa: E402
from paper_2504_18526_gb300 import sisdc as S             # noqa: E402
from tests.helpers import oracle_space                     # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def unpack(theta, n_in, H, q):
    o, p = 0, {}
    for name, shape in (("W1", (n_in, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (H, q)), ("b3", (q,))):
        n = int(np.prod(shape))
        p[name] = theta[o:o + n].reshape(shape).astype(np.float64)
        o += n
    return p


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


CASES = {
    "ns_p5": (dict(pde="ns", dim=2, ncomp=4, gamma=1.4, Re=200.0, Pr=0.72, lo=(0.0, 0.0), hi=(1.0, 1.0),
                   nodes="radau_right", levels=[dict(nel=(9, 7), P=5, M=3)]), 112),
    "burgers_p7": (dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0),
                        nodes="radau_right", levels=[dict(nel=(11, 6), P=7, M=3)]), 64),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tcgen05_forward_matches_mma_sync_and_oracle(dev, case):
    w, H = CASES[case]
    ctx = S.Context(w)
    lv = ctx.levels[0]
    m = S.sisdc_mlp_create(lv, H, seed=5, bf16=1)
    n_in, Hh, q, npar = S.sisdc_mlp_info(m)
    # perturb the biases so that every parameter block is exercised
    theta = np.zeros(npar, dtype=np.float32)
    S.sisdc_mlp_params(m, get=theta)
    rng = np.random.default_rng(21)
    theta = (theta + 0.05 * rng.standard_normal(npar)).astype(np.float32)
    S.sisdc_mlp_params(m, set_=theta)
    sp = oracle_space(w, w["levels"][0])
    r = rng.standard_normal(sp.shape)
    c = 2e-3
    rt = torch.from_numpy(r).to(dev)
    z_tc = torch.zeros(sp.shape, dtype=torch.float64, device=dev)
    z_mma = torch.zeros_like(z_tc)
    S.sisdc_mlp_set_tc(m, True)
    S.sisdc_mlp_apply(m, rt, c, z_tc)
    S.sisdc_mlp_sync(m)
    S.sisdc_mlp_set_tc(m, False)
    S.sisdc_mlp_apply(m, rt, c, z_mma)
    S.sisdc_mlp_sync(m)
    a, b = z_tc.cpu().numpy(), z_mma.cpu().numpy()
    assert np.all(np.isfinite(a))
    # the same BF16 operands, FP32 accumulation in another order
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    p = unpack(theta, n_in, Hh, q)
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    zr = omlp.apply(p, r, sp.nex, sp.ney, q, c, min(sp.hx, sp.hy), round_op=omlp.bf16_round)
    assert np.linalg.norm(a - zr) <= 2e-3 * np.linalg.norm(zr)
    # accumulate mode adds to the output
    S.sisdc_mlp_set_tc(m, True)
    z2 = z_tc.clone()
    S.sisdc_mlp_apply(m, rt, c, z2, add=True)
    S.sisdc_mlp_sync(m)
    assert np.linalg.norm(z2.cpu().numpy() - 2 * a) <= 1e-12 * np.linalg.norm(a)
    S.sisdc_mlp_destroy(m)
    ctx.close()


def test_tcgen05_forward_rejects_unfit_network(dev):
    w, _ = CASES["ns_p5"]
    ctx = S.Context(w)
    m = S.sisdc_mlp_create(ctx.levels[0], 24, seed=1, bf16=1)     # hidden width not a multiple of 16
    with pytest.raises(S.SisdcError) as ei:
        S.sisdc_mlp_set_tc(m, True)
    assert ei.value.status == S.SISDC_E_ARG
    S.sisdc_mlp_destroy(m)
    ctx.close()
