"""The no-allocation solve (sisdc_solve_noalloc) against the allocating one.

Callers that cannot allocate device memory when they need an implicit solve
(a fixed memory budget owned by another framework's allocator, or a loop
that cannot take cudaMalloc's implicit synchronisation) use the entry point
with static scratch.  It must give the same answer as sisdc_solve, on two
calls in a row (the shared scratch array keeps the previous call's
contents), and reject problems that do not fit its fixed array.  This file
is collected last so that a failure here does not hide other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import sisdc as S   # noqa: E402

pytestmark = pytest.mark.gpu

W = dict(pde="burgers", dim=2, ncomp=2, nu=5e-3, lo=(0.0, 0.0), hi=(1.0, 1.0), nodes="radau_right",
         levels=[dict(nel=(12, 10), P=7, M=5)])


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_solve_matches_allocating_solve():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    rtol, maxit = 1e-14, 10000
    ctx = S.Context(W, cg_rtol=rtol, cg_maxit=maxit)
    desc = S.make_level_desc(W, W["levels"][0])
    nc, n, _ = ctx.info(0)
    rng = np.random.default_rng(2504)
    for call, c in enumerate((0.02, 5e-4)):          # two calls in a row
        rhs = torch.from_numpy(rng.standard_normal(nc * n)).to(dev)
        x0 = torch.from_numpy(rng.standard_normal(nc * n)).to(dev)
        x_ref = x0.clone()
        S.sisdc_solve(ctx.levels[0], c, rhs, x_ref)
        S.sisdc_sync(ctx.ctx)
        x_new = x0.clone()
        it = S.sisdc_solve_noalloc(desc, nc, c, rhs, x_new, rtol, maxit)
        torch.cuda.synchronize()
        assert it > 0
        assert _rel(x_new.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-12, call
    ctx.close()


def test_noalloc_allocates_nothing_after_first_call():
    """After a first call on the device (which may commit the static array),
    a further call leaves the device's free memory and PyTorch's reserved
    memory unchanged; a 1D single-component level (the 1D convection-
    diffusion fine level: 16 elements of degree 4) matches sisdc_solve too."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import math
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w1 = dict(pde="convdiff", dim=1, ncomp=1, adv=(1.0, 0.0), nu=0.01, lo=(0.0, 0.0), hi=(2 * math.pi, 0.0),
              nodes="lobatto", levels=[dict(nel=(16, 1), P=4, M=5)])
    ctx = S.Context(w1, cg_rtol=1e-14, cg_maxit=10000)
    desc = S.make_level_desc(w1, w1["levels"][0])
    nc, n, _ = ctx.info(0)
    rng = np.random.default_rng(7)
    rhs = torch.from_numpy(rng.standard_normal(nc * n)).to(dev)
    x0 = torch.from_numpy(rng.standard_normal(nc * n)).to(dev)
    x_ref, xa, xb = x0.clone(), x0.clone(), x0.clone()
    S.sisdc_solve(ctx.levels[0], 0.03, rhs, x_ref)
    S.sisdc_sync(ctx.ctx)
    S.sisdc_solve_noalloc(desc, nc, 0.03, rhs, xa, 1e-14, 10000)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    res0 = torch.cuda.memory_reserved(dev)
    S.sisdc_solve_noalloc(desc, nc, 0.03, rhs, xb, 1e-14, 10000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0 and torch.cuda.memory_reserved(dev) == res0
    for x in (xa, xb):
        assert _rel(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-12
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    dev = torch.device("cuda:0")
    big = dict(W, levels=[dict(nel=(256, 256), P=7, M=5)])
    desc = S.make_level_desc(big, big["levels"][0])
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(S.SisdcError) as ei:
        S.sisdc_solve_noalloc(desc, 2, 0.01, x, x, 1e-12, 100)
    assert ei.value.status == S.SISDC_E_ARG
    assert "too large" in str(ei.value)
