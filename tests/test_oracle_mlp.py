"""Pins for the MLP oracle: finite differences, special cases, textbook Adam, bfloat16."""
import math

import numpy as np

from oracle import mlp_oracle as MO


def data(B=17, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, 6)), rng.standard_normal((B, 2))


def test_param_count():
    assert MO.N_PARAMS == 4738
    th = MO.init_params(1)
    assert np.allclose(MO.pack(MO.unpack(th)), th)


def test_gradient_matches_central_differences():
    X, T = data()
    th = MO.init_params(3)
    th += 0.05 * np.random.default_rng(4).standard_normal(th.size)  # non-zero biases too
    g, _ = MO.grad(th, X, T)
    rng = np.random.default_rng(5)
    for k in rng.choice(th.size, 60, replace=False):
        e = np.zeros_like(th)
        h = 1e-6
        e[k] = h
        fd = (MO.loss(th + e, X, T) - MO.loss(th - e, X, T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_zero_network_outputs_bias_and_loss():
    X, T = data()
    d = MO.unpack(np.zeros(MO.N_PARAMS))
    d["b3"] = np.array([0.3, -0.2])
    th = MO.pack(d)
    y, _ = MO.forward(th, X)
    assert np.allclose(y, [0.3, -0.2])
    assert np.isclose(MO.loss(th, X, T), 0.5 * np.mean(np.sum((T - [0.3, -0.2]) ** 2, 1)))
    g, _ = MO.grad(th, X, T)
    gd = MO.unpack(g)
    assert np.allclose(gd["b3"], np.mean([0.3, -0.2] - T, axis=0))
    assert np.allclose(gd["W1"], 0) and np.allclose(gd["W2"], 0)


def test_adam_first_step_is_sign_step():
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = MO.adam_step(th, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(new, th - 0.01 * np.sign(g), atol=1e-7)


def test_adam_three_steps_hand_worked():
    """Adam (Kingma & Ba, Algorithm 1; beta1 0.9, beta2 0.999, eps 1e-8) on one parameter with
    gradients +1, -1, +2, worked by hand from the definition:
      t=1: m = 1/10, v = 1/1000;        m^ = 1,        v^ = 1
      t=2: m = -1/100, v = 1999/1e6;    m^ = -1/19,    v^ = 1999/1999 = 1
      t=3: m = 191/1000, v = 5997001/1e9; m^ = 191/271, v^ = 5997001/2997001
    (1 - 0.9^2 = 19/100, 1 - 0.9^3 = 271/1000, 1 - 0.999^3 = 2997001/1e9). A moment update or a
    bias correction that is right only at t = 1 fails steps 2 and 3."""
    lr, eps = 0.1, 1e-8
    steps = [lr * 1.0 / (1.0 + eps),
             lr * (-1.0 / 19.0) / (1.0 + eps),
             lr * (191.0 / 271.0) / (math.sqrt(5997001.0 / 2997001.0) + eps)]
    th, m, v = np.array([0.5]), np.zeros(1), np.zeros(1)
    want = 0.5
    for t, (g, step) in enumerate(zip([1.0, -1.0, 2.0], steps), start=1):
        th, m, v = MO.adam_step(th, np.array([g]), m, v, t, lr=lr)
        want -= step
        assert abs(th[0] - want) < 1e-14, (t, th[0], want)
    assert abs(m[0] - 0.191) < 1e-15 and abs(v[0] - 5997001e-9) < 1e-17


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 65504.0])
    r = MO.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == 1.0 + 2 ** -6
    assert r[4] == -2.5


def test_training_by_gradient_descent_reduces_loss():
    X, _ = data(64, 1)
    teacher = MO.init_params(9)
    T, _ = MO.forward(teacher, X)
    th = MO.init_params(10)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = MO.loss(th, X, T)
    for t in range(1, 201):
        g, _ = MO.grad(th, X, T)
        th, m, v = MO.adam_step(th, g, m, v, t, lr=3e-3)
    assert MO.loss(th, X, T) < 0.1 * l0
