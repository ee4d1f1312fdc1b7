"""Pins of the cost model's FP64 oracle (CPU).

The analytic gradient is checked against central finite differences (an
independent computation of the same derivative), the forward pass against
networks whose output is known in closed form, and Adam against its first
step, which the definition fixes to -lr * g / (|g| + eps) per coordinate.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(scale=scale, size=M.NPARAMS)


def random_data(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, M.NF))
    T = rng.normal(size=n)
    return X, T


def test_layout_size():
    assert M.NPARAMS == 52 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 7617
    p = np.arange(M.NPARAMS, dtype=np.float64)
    assert np.array_equal(M.pack(*M.unpack(p)), p)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_finite_differences(seed):
    p = random_params(seed)
    X, T = random_data(seed + 10)
    g = M.gradient(p, X, T)
    rng = np.random.default_rng(seed)
    idx = list(rng.choice(M.NPARAMS, 60, replace=False)) + [M.NPARAMS - 1, 0, 52 * 64 + 3]
    fd = M.finite_difference(p, X, T, idx)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-9)


def test_forward_closed_form():
    """With W1 = copy of the first 64 inputs, identity W2, W3 = 1 and zero
    biases the output is the sum of the positive first 64 inputs."""
    W1 = np.zeros((M.NF, M.H))
    for j in range(min(M.NF, M.H)):
        W1[j, j] = 1.0
    p = M.pack(W1, np.zeros(M.H), np.eye(M.H), np.zeros(M.H), np.ones(M.H), 0.25)
    X = np.random.default_rng(4).normal(size=(7, M.NF))
    y, _ = M.forward(p, X)
    want = np.where(X[:, :M.H] > 0, X[:, :M.H], 0).sum(axis=1) + 0.25
    assert np.allclose(y, want, rtol=0, atol=1e-12)


def test_relu_kink_convention():
    """ReLU'(0) = 0: a unit sitting exactly at z = 0 passes no gradient."""
    W1 = np.zeros((M.NF, M.H))
    p = M.pack(W1, np.zeros(M.H), np.eye(M.H), np.zeros(M.H), np.ones(M.H), 0.0)
    X = np.ones((3, M.NF))
    g = M.gradient(p, X, np.ones(3))
    W1g, b1g, *_ = M.unpack(g)
    assert np.all(W1g == 0) and np.all(b1g == 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = M.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_adam_minimises_a_quadratic():
    p, m, v = np.array([3.0, -2.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        p, m, v = M.adam_step(p, m, v, 2 * p, t, lr=0.01)
    assert np.all(np.abs(p) < 1e-3)


def test_planted_gradient_mistake_is_caught():
    """A gradient with the ReLU mask dropped on layer 1 fails the check."""
    p = random_params(7)
    X, T = random_data(8)
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    y, (Xd, z1, h1, z2, h2) = M.forward(p, X)
    dy = 2.0 * (y - T) / y.size
    dz2 = np.outer(dy, W3) * (z2 > 0)
    dz1_wrong = dz2 @ W2.T
    gW1_wrong = Xd.T @ dz1_wrong
    idx = list(range(0, 52 * 64, 97))
    fd = M.finite_difference(p, X, T, idx)
    assert not np.allclose(np.ravel(gW1_wrong)[idx], fd, rtol=1e-3, atol=1e-7)
