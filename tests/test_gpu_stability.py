"""Batched stability function R(z) of one SI-MLSDC step on the Dahlquist
problem (Sec. 5), one GPU thread per point, against the oracle's step of
the same scalar problem (relative 1e-12), for single-level SDC, Cascade,
FMG (C_fmg = 1, 2), Lobatto nodes and SI(1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_18526_gb300 import sisdc as S          # noqa: E402
from oracle.dahlquist import stability                  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    S.load()
    return torch.device("cuda:0")


CASES = [
    dict(Ms=[5], nodes="radau_right", stages=2, ncycles=3, start="predictor"),
    dict(Ms=[3, 5], nodes="radau_right", stages=2, ncycles=2, start="cascade"),
    dict(Ms=[2, 3, 5], nodes="radau_right", stages=2, ncycles=2, start="fmg1", fmg_cycles=1),
    dict(Ms=[2, 3, 5], nodes="radau_right", stages=2, ncycles=1, start="fmg1", fmg_cycles=2),
    dict(Ms=[3, 5], nodes="lobatto", stages=2, ncycles=2, start="predictor"),
    dict(Ms=[3, 5], nodes="radau_right", stages=1, ncycles=2, start="predictor", post_sweep=False),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_stability_map_matches_oracle(dev, k):
    case = dict(CASES[k])
    rng = np.random.default_rng(100 + k)
    z = rng.uniform(-30.0, 2.0, 64) + 1j * rng.uniform(-20.0, 20.0, 64)
    z[:4] = [0.0, -1.0, 1j, -5.0 + 5.0j]
    Rg = S.sisdc_stability(torch.from_numpy(z).to(dev), **case).cpu().numpy()
    fmg_cycles = case.pop("fmg_cycles", 1)
    post = case.pop("post_sweep", True)
    Ro = np.array([stability(zz, case["Ms"], case["nodes"], case["stages"], case["ncycles"], case["start"],
                             post_sweep=post, fmg_cycles=fmg_cycles) for zz in z])
    assert np.all(np.abs(Rg - Ro) <= 1e-12 * np.maximum(1.0, np.abs(Ro)))
    assert abs(Rg[0] - 1.0) < 1e-14      # z = 0: u stays 1
