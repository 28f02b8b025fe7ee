"""Failure detection of the bounded grid barrier, without a GPU fault.

Every persistent kernel synchronises its blocks through a grid barrier whose
wait is bounded; a block whose wait runs out records a timeout for the host
and leaves the kernel.  sisdc_barrier_selftest launches one barrier that one
block never reaches (an arrival that nothing makes), so the other blocks'
wait runs out after a short limit; the host must read SISDC_E_TIMEOUT and the
context must stay usable for the method's own kernels afterwards.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import inputs, sisdc as S   # noqa: E402
from tests.helpers import oracle_space                   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return S.load()


def test_barrier_completes_when_every_block_arrives(lib):
    assert lib.sisdc_barrier_selftest(8, -1, 200.0, None) == S.SISDC_OK
    assert lib.sisdc_barrier_selftest(torch.cuda.get_device_properties(0).multi_processor_count, -1, 200.0,
                                      None) == S.SISDC_OK


def test_barrier_timeout_reported_and_context_usable(lib):
    t0 = time.perf_counter()
    st = lib.sisdc_barrier_selftest(8, 3, 200.0, None)
    el = time.perf_counter() - t0
    assert st == S.SISDC_E_TIMEOUT
    assert 0.15 < el < 10.0
    # the barrier words were reset by the last block out: the next launch completes
    assert lib.sisdc_barrier_selftest(8, -1, 200.0, None) == S.SISDC_OK
    # and the method's persistent kernels still run on this context
    w = inputs.scaled("burgers2d", nel=(4, 4))
    X, Y = oracle_space(w, w["levels"][-1]).coords()
    u0 = inputs.burgers2d_initial(X, Y)
    ctx = S.Context(w)
    du = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    S.sisdc_step(ctx.ctx, du, 0.0, 1e-4, 2, S.START_IDS["cascade"], 1)
    S.sisdc_sync(ctx.ctx)
    ctx.close()
    assert torch.isfinite(du).all()


def test_barrier_selftest_rejects_bad_arguments(lib):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert lib.sisdc_barrier_selftest(0, -1, 200.0, None) == S.SISDC_E_ARG
    assert lib.sisdc_barrier_selftest(nsm + 1, -1, 200.0, None) == S.SISDC_E_ARG
    assert lib.sisdc_barrier_selftest(8, 8, 200.0, None) == S.SISDC_E_ARG
    assert lib.sisdc_barrier_selftest(8, -1, 0.0, None) == S.SISDC_E_ARG
    assert lib.sisdc_barrier_selftest(8, -1, 5000.0, None) == S.SISDC_E_ARG
