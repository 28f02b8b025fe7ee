"""Caller-owned allocator for the level work arrays (sisdc_set_allocator):
with PyTorch's caching allocator the level memory is part of torch's pool,
the results equal those of the default allocator bit for bit, everything is
returned at sisdc_destroy, and allocator failures and misuse are reported
as statuses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S   # noqa: E402
from tests.helpers import oracle_space                   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


def _burgers(nel=6):
    w = inputs.scaled("burgers2d", nel=(nel, nel))
    X, Y = oracle_space(w, w["levels"][-1]).coords()
    u0 = inputs.burgers2d_initial(X, Y)
    dt = inputs.cfl_dt(0.5, 1.0 / nel, 7, inputs.max_wave_speed("burgers", u0))
    return w, u0, dt


def _run(w, u0, dt, dev, allocator=None):
    ctx = S.Context(w, allocator=allocator, cg_rtol=1e-12)
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    for n in range(2):
        S.sisdc_step(ctx.ctx, du, n * dt, dt, 3, S.START_IDS["cascade"], 1)
    S.sisdc_sync(ctx.ctx)
    return ctx, du.cpu().numpy()


def test_torch_allocator_owns_level_memory(dev):
    w, u0, dt = _burgers()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ref_ctx, ref = _run(w, u0, dt, dev)
    ref_ctx.close()
    alloc = S.TorchAllocator()
    ctx, out = _run(w, u0, dt, dev, alloc)
    held = torch.cuda.memory_allocated() - base
    assert len(alloc.live) == 2 * len(w["levels"])          # tables and work arrays per level
    assert held >= sum(alloc.live.values()) > 0
    assert np.array_equal(out, ref)
    ctx.close()
    torch.cuda.synchronize()
    assert not alloc.live
    assert torch.cuda.memory_allocated() == base


def test_allocator_failure_and_misuse(dev):
    w, u0, dt = _burgers(4)
    ctx = S.sisdc_create(S.make_problem(w))
    failing = type("Failing", (), {})()
    failing.alloc = S.ALLOC_FN(lambda n, s, u: None)
    failing.release = S.RELEASE_FN(lambda p, n, s, u: None)
    S.sisdc_set_allocator(ctx, failing)
    with pytest.raises(S.SisdcError) as ei:
        S.sisdc_create_level(ctx, S.make_level_desc(w, w["levels"][0]))
    assert ei.value.status == S.SISDC_E_OOM
    # the context is still usable: back to cudaMalloc, levels, a step
    S.sisdc_set_allocator(ctx, None)
    for lv in w["levels"]:
        S.sisdc_create_level(ctx, S.make_level_desc(w, lv))
    with pytest.raises(S.SisdcError) as ei:                   # too late once a level exists
        S.sisdc_set_allocator(ctx, S.TorchAllocator())
    assert ei.value.status == S.SISDC_E_STATE
    du = torch.from_numpy(np.ascontiguousarray(u0)).to(dev)
    S.sisdc_step(ctx, du, 0.0, dt, 2, S.START_IDS["cascade"], 1)
    S.sisdc_sync(ctx)
    assert torch.isfinite(du).all()
    S.sisdc_destroy(ctx)
