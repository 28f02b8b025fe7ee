"""Pins for the oracle's element-patch MLP (CPU only): gradients against
central finite differences, patch gathering against direct indexing."""
import numpy as np

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
