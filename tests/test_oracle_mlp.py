"""Pins for the MLP oracle: gradients against central differences, BF16 rounding
against its definition, Adam against hand-evaluated steps (first step, three
steps with distinct betas, and the unrolled moment sums), and the moment mode
list against its ordering rule."""
import numpy as np
import pytest

from oracle import mlp as M


def small(seed=0, hidden=16, B=12):
    rng = np.random.default_rng(seed)
    p = M.init_params(hidden, seed)
    for k in ("b1", "b2"):
        p[k] = rng.normal(0, 0.1, size=p[k].shape)
    p["b3"] = np.array([0.3])
    X = rng.normal(size=(B, M.IN_FEATURES))
    t = rng.normal(size=B)
    return p, X, t


def test_gradients_match_central_differences():
    p, X, t = small()
    _, g = M.loss_and_grads(p, X, t)
    h = 1e-6
    rng = np.random.default_rng(3)
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = M.loss_and_grads(p, X, t)
            flat[idx] = old - h
            lm, _ = M.loss_and_grads(p, X, t)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(num, rel=1e-5, abs=1e-8), (k, idx)


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.14159, 0.0, 65504.0])
    got = M.bf16(vals)
    # BF16 keeps 8 significant bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -7 and got[3] == 1.0 + 2 ** -6
    assert got[4] == pytest.approx(-3.140625) and got[5] == 0.0
    assert np.all(np.abs(got - vals) <= np.abs(vals) * 2 ** -8)


def test_adam_first_step_moves_by_lr_sign():
    # With bias correction the first step is -lr * g / (|g| + eps) = -lr * sign(g).
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3])}
    M.adam_step(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["a"], [0.99, -1.99, 0.49], atol=1e-6)


def test_adam_three_steps_hand_evaluated():
    # Kingma & Ba, Algorithm 1, evaluated by hand for one scalar with beta1 = 1/2,
    # beta2 = 3/4 (distinct, so a swap changes the answer), lr = 0.1, eps = 0 and
    # gradients 1, -2, 3 from theta0 = 1:
    #   t=1: m = 1/2,  v = 1/4;      m^ = 1,          v^ = 1          -> step -0.1
    #   t=2: m = -3/4, v = 19/16;    m^ = -1,         v^ = 19/7       -> step +0.1 / sqrt(19/7)
    #   t=3: m = 9/8,  v = 201/64;   m^ = 9/7,        v^ = 201/37     -> step -0.1 (9/7) / sqrt(201/37)
    expected = [0.9, 0.9 + 0.1 / np.sqrt(19 / 7)]
    expected.append(expected[-1] - 0.1 * (9 / 7) / np.sqrt(201 / 37))
    p = {"a": np.array([1.0])}
    st = {}
    for g, want in zip((1.0, -2.0, 3.0), expected):
        M.adam_step(p, {"a": np.array([g])}, st, lr=0.1, beta1=0.5, beta2=0.75, eps=0.0)
        assert p["a"][0] == pytest.approx(want, rel=1e-14), (st["t"], p["a"][0], want)
    assert st["t"] == 3
    # the same updates with the betas swapped or without bias correction end elsewhere
    assert abs(expected[-1] - 0.905535) < 1e-6
    p2, st2 = {"a": np.array([1.0])}, {}
    for g in (1.0, -2.0, 3.0):
        M.adam_step(p2, {"a": np.array([g])}, st2, lr=0.1, beta1=0.75, beta2=0.5, eps=0.0)
    assert abs(p2["a"][0] - expected[-1]) > 1e-4
    no_bias_corr_t2 = 0.9 + 0.1 * (3 / 4) / np.sqrt(19 / 16)  # step 2 without the corrections
    assert abs(no_bias_corr_t2 - expected[1]) > 1e-3


def test_adam_matches_closed_form_moment_sums():
    # After t steps m_t = (1 - b1) sum_s b1^(t-s) g_s and v_t = (1 - b2) sum_s b2^(t-s) g_s^2
    # (the recurrences unrolled); every step divides their bias-corrected ratio.
    rng = np.random.default_rng(11)
    b1, b2, lr, eps = 0.9, 0.999, 1e-2, 1e-8
    gs = rng.normal(size=(5, 7)) * np.array([1e-3, 1e-2, 0.1, 1, 10, 100, 1e3])
    p = {"w": rng.normal(size=7)}
    theta = p["w"].copy()
    st = {}
    for t in range(1, 6):
        M.adam_step(p, {"w": gs[t - 1]}, st, lr=lr, beta1=b1, beta2=b2, eps=eps)
        m = (1 - b1) * sum(b1 ** (t - s) * gs[s - 1] for s in range(1, t + 1))
        v = (1 - b2) * sum(b2 ** (t - s) * gs[s - 1] ** 2 for s in range(1, t + 1))
        theta = theta - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        np.testing.assert_allclose(p["w"], theta, rtol=1e-12, atol=1e-15)


def test_moment_modes_ordering():
    m = M.moment_modes(32, 64)
    assert m.shape == (64, 3)
    q = (m ** 2).sum(axis=1)
    assert np.all(np.diff(q) >= 0)
    assert np.all(m[:, 2] >= 0) and not np.any(np.all(m == 0, axis=1))
    assert q[0] == 1 and sum(q == 1) == 5  # (-1,0,0), (0,-1,0), (0,0,1), (0,1,0), (1,0,0)
    assert tuple(m[0]) == (-1, 0, 0)


def test_features_layout():
    q = np.array([[-0.5, 0.5, 0.5, 0.5], [2.0, 0.0, 0.0, 0.0]])
    fa, fb = np.arange(64) / 64.0, -np.arange(64) / 64.0
    X = M.features(q, fa, fb)
    assert X.shape == (2, 132)
    np.testing.assert_allclose(X[0, :4], [0.5, -0.5, -0.5, -0.5])
    np.testing.assert_allclose(X[1, :4], [1, 0, 0, 0])
    np.testing.assert_allclose(X[:, 4:68], np.broadcast_to(fa, (2, 64)))
