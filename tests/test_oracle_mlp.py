"""Pins for the oracle's element-patch MLP (CPU only): gradients against
central finite differences, patch gathering against direct indexing,
the bfloat16 rounding of the BF16 mode against closed forms and PyTorch."""
import numpy as np
import pytest

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(13, 7, 5, seed=1)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((11, 13))
    T = rng.standard_normal((11, 5))
    _, g = mlp.loss_and_grads(p, X, T)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp.loss_and_grads(p, X, T)
            flat[idx] = old - eps
            lm, _ = mlp.loss_and_grads(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd))


def test_patches_direct_indexing():
    rng = np.random.default_rng(2)
    nc, ney, nex, q = 2, 3, 4, 5
    f = rng.standard_normal((nc, ney, nex, q))
    rows, s = mlp.patches(f, nex, ney, q, c=0.3, h=0.5)
    r = 0
    for c in range(nc):
        for ey in range(ney):
            for ex in range(nex):
                raw = np.concatenate([f[c, (ey + dy) % ney, (ex + dx) % nex]
                                      for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
                sc = np.sqrt(np.mean(raw ** 2))
                assert abs(s[r] - sc) < 1e-14
                assert np.allclose(rows[r, :9 * q], raw / sc, atol=1e-14)
                assert abs(rows[r, -1] - 0.1 * np.log(0.3 / 0.25)) < 1e-14
                r += 1


def test_training_reduces_loss_on_a_linear_target():
    """Plain gradient descent with the oracle gradients fits a linear map."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((64, 10))
    A = rng.standard_normal((10, 4)) * 0.3
    T = X @ A
    p = mlp.init_params(10, 16, 4, seed=4)
    l0, _ = mlp.loss_and_grads(p, X, T)
    for _ in range(300):
        _, g = mlp.loss_and_grads(p, X, T)
        for k in p:
            p[k] -= 0.5 * g[k]
    l1, _ = mlp.loss_and_grads(p, X, T)
    assert l1 < 0.2 * l0


def test_bf16_round_closed_forms_and_library():
    """bf16_round: ties to even at closed-form halfway points, exact on values
    that fit 8 bits, overflow to infinity, and the same bits as PyTorch's
    bfloat16 conversion on random float32 values."""
    from oracle.mlp import bf16_round
    assert bf16_round(1.0 + 2.0 ** -8) == 1.0                       # tie, even neighbour 1.0
    assert bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie, rounds up to even
    assert bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert bf16_round(-(1.0 + 2.0 ** -9)) == -1.0
    assert bf16_round(1.5) == 1.5 and bf16_round(0.0) == 0.0 and bf16_round(-3.0 * 2.0 ** -100) == -3.0 * 2.0 ** -100
    assert np.isinf(bf16_round(3.4e38))
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-30, 30, 100000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(x), ref)


def test_round_op_identity_is_the_plain_network():
    """With round_op = None the forward pass and gradients are the plain FP64
    network (the form pinned by finite differences above), and rounding every
    operand to bfloat16 moves them by the size of one bfloat16 rounding."""
    from oracle import mlp as M
    rng = np.random.default_rng(9)
    p = M.init_params(12, 8, 4, 3)
    X = rng.standard_normal((20, 12))
    T = rng.standard_normal((20, 4))
    l0, g0 = M.loss_and_grads(p, X, T)
    l1, g1 = M.loss_and_grads(p, X, T, round_op=lambda a: a)
    assert l0 == l1 and all(np.array_equal(g0[k], g1[k]) for k in g0)
    lb, gb = M.loss_and_grads(p, X, T, round_op=M.bf16_round)
    rel = np.linalg.norm(gb["W1"] - g0["W1"]) / np.linalg.norm(g0["W1"])
    assert 1e-5 < rel < 3e-2 and abs(lb - l0) < 3e-2 * abs(l0)
