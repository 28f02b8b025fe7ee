"""FP64 reference of the element-patch MLP (test infrastructure only).

The learned part of the implicit stage (not in the paper; an addition that
leaves the method unchanged): for every element and component, the 3x3 element patch of a
residual field r (9 Q nodal values, ordered by neighbour offset (dy, dx) in
{-1, 0, 1}^2 row-major, each element's nodes in the state layout) is scaled
by its RMS s, a scalar feature 0.1 log(c / h^2) is appended, and a 3-layer
perceptron with tanh hidden activations predicts the deviation of the
centre element's correction from the residual itself (the exact correction
when c -> 0), scaled back by s:
    z = r_centre + s * MLP([r_patch / s, 0.1 log(c / h^2)]).
Loss: mean over samples of 0.5 * mean_q (MLP(x) - t)^2 with
t = (dx - r_centre) / s.

The optional round_op is applied to both operands of every matrix product
(the BF16 mode of the CUDA kernels rounds them to bfloat16 as it stages them
for the tensor cores; sums, biases and tanh stay in full precision).

Pins (tests/test_oracle_mlp.py): gradients against central finite
differences; patch gathering against direct indexing on a small mesh;
bf16_round against closed-form ties and the bfloat16 conversion of PyTorch.
"""
import numpy as np


def init_params(n_in, hidden, n_out, seed):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((n_in, hidden)) / np.sqrt(n_in)
    W2 = rng.standard_normal((hidden, hidden)) / np.sqrt(hidden)
    W3 = rng.standard_normal((hidden, n_out)) / np.sqrt(hidden) * 0.1
    return {"W1": W1, "b1": np.zeros(hidden), "W2": W2, "b2": np.zeros(hidden),
            "W3": W3, "b3": np.zeros(n_out)}


def bf16_round(a):
    """Nearest bfloat16 value (8 significand bits, ties to even) of a, taken
    through its float32 bit pattern: add 0x7FFF plus the lowest kept bit to
    the pattern, then clear the 16 dropped bits."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def forward(p, X, round_op=None):
    R = round_op or _ident
    h1 = np.tanh(R(X) @ R(p["W1"]) + p["b1"])
    h2 = np.tanh(R(h1) @ R(p["W2"]) + p["b2"])
    y = R(h2) @ R(p["W3"]) + p["b3"]
    return y, (X, h1, h2)


def loss_and_grads(p, X, T, round_op=None):
    """0.5 * mean over samples and outputs of (y - t)^2, and its gradients."""
    R = round_op or _ident
    y, (X, h1, h2) = forward(p, X, round_op)
    n, q = T.shape
    d = (y - T) / (n * q)
    loss = 0.5 * np.sum((y - T) ** 2) / (n * q)
    g = {"W3": R(h2).T @ R(d), "b3": d.sum(axis=0)}
    dh2 = (R(d) @ R(p["W3"]).T) * (1.0 - h2 * h2)
    g["W2"] = R(h1).T @ R(dh2)
    g["b2"] = dh2.sum(axis=0)
    dh1 = (R(dh2) @ R(p["W2"]).T) * (1.0 - h1 * h1)
    g["W1"] = R(X).T @ R(dh1)
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def patches(field, nex, ney, q, c, h):
    """Rows [ncomp*nel, 9q + 1] of RMS-scaled 3x3 element patches of a state
    field[ncomp][ney][nex][q] (periodic), and the scales s [ncomp*nel]."""
    f = np.asarray(field).reshape(-1, ney, nex, q)
    nc = f.shape[0]
    rows = np.empty((nc, ney, nex, 9 * q + 1))
    for k, (dy, dx) in enumerate([(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]):
        rows[..., k * q:(k + 1) * q] = np.roll(np.roll(f, -dy, axis=1), -dx, axis=2)
    s = np.sqrt(np.mean(rows[..., :9 * q] ** 2, axis=-1))
    s = np.where(s > 0, s, 1.0)
    rows[..., :9 * q] /= s[..., None]
    rows[..., 9 * q] = 0.1 * np.log(c / (h * h))
    return rows.reshape(nc * ney * nex, 9 * q + 1), s.reshape(-1)


def targets(field, dx, s, q):
    """t = (dx - r_centre) / s per row."""
    return (np.asarray(dx).reshape(-1, q) - np.asarray(field).reshape(-1, q)) / s[:, None]


def apply(p, field, nex, ney, q, c, h, round_op=None):
    """z = r_centre + s * MLP(patch / s) for every element and component."""
    X, s = patches(field, nex, ney, q, c, h)
    y, _ = forward(p, X, round_op)
    return (np.asarray(field).reshape(-1, q) + y * s[:, None]).reshape(np.shape(field))
