"""Pins of the FP64 surrogate oracle (forward pass, backpropagated gradient,
Adam) against values fixed by mathematics rather than by the oracle itself."""
import numpy as np

import workloads as W
from oracle import mlp as M


def _rand_problem(n=6, seed=3, scale=1.0):
    r = np.random.default_rng(seed)
    th = W.mlp_init(20) * scale
    th[M.OFF["b1"]:M.OFF["b1"] + 128] = r.normal(0, 0.3, 128)
    th[M.OFF["b2"]:M.OFF["b2"] + 128] = r.normal(0, 0.3, 128)
    th[M.OFF["b3"]:M.OFF["b3"] + 6] = r.normal(0, 0.3, 6)
    x = r.normal(0, 1, (n, 2))
    t = r.normal(0, 1, (n, 6))
    return th, x, t


def test_gradient_matches_central_differences():
    """Backpropagation against (L(theta + h e_k) - L(theta - h e_k)) / 2h on
    parameters of every block; the difference quotient's error is O(h^2)."""
    th, x, t = _rand_problem()
    loss, g = M.loss_grad(th, x, t)
    r = np.random.default_rng(9)
    ks = []
    for name, shape in M.SHAPES.items():
        size = int(np.prod(shape))
        ks += list(M.OFF[name] + r.choice(size, min(size, 24), replace=False))
    for k in ks:
        h = 1e-5
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_grad(tp, x, t)[0] - M.loss_grad(tm, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3), (k, fd, g[k])


def test_saturated_network_is_an_integer_product():
    """With |pre-activations| >= 30 every tanh rounds to +-1 exactly, so the
    output is y = W3 sign(A s + 1/2) + b3 in integers: pins the wiring of
    every layer (which index multiplies which, biases, layer order)."""
    r = np.random.default_rng(4)
    s = r.choice([-1.0, 1.0], 128)
    A = r.integers(-2, 3, (128, 128)).astype(float)
    W3 = r.integers(-3, 4, (6, 128)).astype(float)
    b3 = r.integers(-5, 6, 6).astype(float)
    th = M.pack(dict(W1=np.zeros((128, 2)), b1=60.0 * s, W2=60.0 * A, b2=np.full(128, 30.0), W3=W3, b3=b3))
    y = M.forward(th, np.array([[0.3, -1.2], [2.0, 0.5]]))
    h2 = np.sign(A @ s + 0.5)
    expect = W3 @ h2 + b3
    assert np.array_equal(y[0], expect) and np.array_equal(y[1], expect)
    # the transposed weight would give a different sign pattern
    assert not np.array_equal(W3 @ np.sign(A.T @ s + 0.5) + b3, expect)


def test_hidden_sign_symmetry():
    """tanh is odd: negating W1, b1 and the columns of W2 leaves the output
    unchanged; negating b3 does not."""
    th, x, _ = _rand_problem()
    p = M.unpack(th)
    q = dict(p)
    q["W1"], q["b1"], q["W2"] = -p["W1"], -p["b1"], -p["W2"]
    assert np.allclose(M.forward(M.pack(q), x), M.forward(th, x), rtol=0, atol=1e-13)


def test_adam_first_steps_closed_form():
    """From m = v = 0 the bias-corrected moments are g and g^2 for a constant
    gradient, so each of the first steps moves theta by lr g / (|g| + eps)."""
    r = np.random.default_rng(5)
    th0 = r.normal(size=M.N_PARAMS)
    g = r.normal(size=M.N_PARAMS) * np.exp(r.uniform(-8, 2, M.N_PARAMS))
    th, m, v = th0.copy(), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    lr, eps = 1e-3, 1e-8
    for step in (1, 2, 3):
        M.adam(th, m, v, g, step, lr=lr, eps=eps)
        expect = th0 - step * lr * g / (np.abs(g) + eps)
        assert np.allclose(th, expect, rtol=1e-12, atol=1e-15)


def test_training_reduces_loss_on_a_smooth_target():
    """Full-batch Adam fits six smooth functions of two inputs."""
    r = np.random.default_rng(6)
    x = r.uniform(-1, 1, (32, 2))
    t = np.stack([np.sin(2 * x[:, 0]), x[:, 1] ** 2, x[:, 0] * x[:, 1], np.cos(x[:, 1]), x[:, 0], -x[:, 1]], 1)
    th = W.mlp_init(21)
    m, v = np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    l0, _ = M.loss_grad(th, x, t)
    M.train(th, m, v, 0, x, t, 300, lr=3e-3)
    l1, _ = M.loss_grad(th, x, t)
    assert l1 < 0.02 * l0, (l0, l1)
