"""FP64 oracle for the learned rotation proposal (not part of the paper).

TEST INFRASTRUCTURE ONLY: imported by the test suite and the benchmark's CPU
legs, never by the product path.  Plain NumPy, written from the definitions:

* features: x = [q (unit, w >= 0); |f_A(m_i)| / f_A(0), i < 64; |f_B(m_i)| / f_B(0), i < 64]
  with m_1..m_64 the lowest modes of the half spectrum (m_z >= 0, m != 0,
  components in (-N/2, N/2)) ordered by (|m|^2, m_x, m_y, m_z); B unrotated;
* network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3
  (132 -> H -> H -> 1);
* loss: mean squared error; gradients by the chain rule; Adam (Kingma & Ba,
  2015) with bias correction.

`bf16=True` rounds the quantities the GPU keeps in BF16 (weights, inputs,
hidden activations and hidden gradients) to BF16, round-to-nearest-even, so
that the comparison isolates accumulation order.  Pinned by central
differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

IN_FEATURES = 132


def moment_modes(N: int, count: int = 64):
    """The `count` lowest modes of the half spectrum, ordered by (|m|^2, m_x, m_y, m_z)."""
    h = N // 2
    modes = []
    for mx in range(-h + 1, h):
        for my in range(-h + 1, h):
            for mz in range(0, h):
                if mx == 0 and my == 0 and mz == 0:
                    continue
                modes.append((mx * mx + my * my + mz * mz, mx, my, mz))
    modes.sort()
    return np.array([m[1:] for m in modes[:count]], dtype=np.int64)


def moments(spectrum: np.ndarray, modes: np.ndarray) -> np.ndarray:
    """|f(m)| / f(0) on a half spectrum stored [ix][iy][iz] in FFT order (complex)."""
    N = spectrum.shape[0]
    ix = modes[:, 0] % N
    iy = modes[:, 1] % N
    return np.abs(spectrum[ix, iy, modes[:, 2]]) / spectrum[0, 0, 0].real


def canonical_quats(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    return np.where(q[:, :1] < 0, -q, q)


def features(q, fa, fb) -> np.ndarray:
    q = canonical_quats(q)
    n = q.shape[0]
    return np.concatenate([q, np.broadcast_to(fa, (n, fa.size)), np.broadcast_to(fb, (n, fb.size))], axis=1)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return rounded.view(np.float32).astype(np.float64)


def init_params(hidden: int, seed: int):
    """He-uniform initial weights from a seeded generator (biases zero)."""
    rng = np.random.default_rng(seed)

    def u(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape)

    return {"W1": u(IN_FEATURES, (hidden, IN_FEATURES)), "b1": np.zeros(hidden),
            "W2": u(hidden, (hidden, hidden)), "b2": np.zeros(hidden),
            "w3": u(hidden, (hidden,)), "b3": np.zeros(1)}


def forward(p, X, bf=False):
    r = bf16 if bf else (lambda a: a)
    X = r(X)
    z1 = X @ r(p["W1"]).T + p["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ r(p["w3"]) + p["b3"][0]
    return y, (X, h1, h2)


def loss_and_grads(p, X, t, bf=False):
    """Mean squared error and its gradients with respect to every parameter."""
    r = bf16 if bf else (lambda a: a)
    y, (Xr, h1, h2) = forward(p, X, bf)
    B = X.shape[0]
    d = y - t
    loss = float(np.mean(d * d))
    gy = 2.0 * d / B
    g = {"w3": h2.T @ gy, "b3": np.array([gy.sum()])}
    dh2 = r(np.outer(gy, r(p["w3"])) * (h2 > 0))
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = r((dh2 @ r(p["W2"])) * (h1 > 0))
    g["W1"] = dh1.T @ Xr
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v per parameter and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
