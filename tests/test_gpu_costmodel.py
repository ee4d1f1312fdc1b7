"""Cost-model kernels against the FP64 oracle (GPU).

The forward pass, the gradient of the mean squared error and one Adam step
are compared with oracle/mlp_oracle.py on seeded data whose sample count
spans several 64-sample chunks and CTAs and ends in a ragged chunk.
Tolerances follow from FP32 arithmetic: outputs within 1e-4 relative to
their scale, gradients within 1e-3 relative error in the 2-norm.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_15098_gb300 import build as B
    B.build()
    from paper_2605_15098_gb300 import sv as mod
    return mod


def data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, M.NF)).astype(np.float32)
    T = rng.normal(size=n).astype(np.float32)
    return X, T


def model_with(sv, p):
    m = sv.sv_cost_model_create(1)
    sv.sv_cost_model_set_params(m, p)
    return m


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 20001])
def test_forward_matches_oracle(sv, n):
    rng = np.random.default_rng(n)
    p = (rng.normal(scale=0.2, size=M.NPARAMS)).astype(np.float32)
    X, _ = data(n + 1, n)
    m = model_with(sv, p)
    try:
        y = sv.sv_cost_model_predict(m, X)
    finally:
        sv.sv_cost_model_destroy(m)
    want, _ = M.forward(p.astype(np.float64), X.astype(np.float64))
    scale = max(1.0, float(np.max(np.abs(want))))
    assert np.max(np.abs(y - want)) <= 1e-4 * scale


@pytest.mark.parametrize("n", [5, 64, 777, 5000])
def test_gradient_matches_oracle(sv, n):
    rng = np.random.default_rng(10 + n)
    p = (rng.normal(scale=0.2, size=M.NPARAMS)).astype(np.float32)
    X, T = data(20 + n, n)
    m = model_with(sv, p)
    try:
        g, loss = sv.sv_cost_model_gradient(m, X, T)
    finally:
        sv.sv_cost_model_destroy(m)
    p64, X64, T64 = p.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    want = M.gradient(p64, X64, T64)
    rel = np.linalg.norm(g - want) / np.linalg.norm(want)
    assert rel <= 1e-3, rel
    assert abs(loss - M.loss(p64, X64, T64)) <= 1e-4 * max(1.0, M.loss(p64, X64, T64))
    # each layer separately, so that a wrong small block is not hidden
    parts = [(0, 52 * 64), (52 * 64, 52 * 64 + 64), (3392, 3392 + 4096), (7488, 7552),
             (7552, 7616), (7616, 7617)]
    for a, b in parts:
        ra = np.linalg.norm(g[a:b] - want[a:b]) / max(np.linalg.norm(want[a:b]), 1e-30)
        assert ra <= 2e-3 or np.linalg.norm(want[a:b]) < 1e-7, (a, b, ra)


def test_adam_step_matches_oracle(sv):
    """One epoch with one full batch = one Adam step from zero moments."""
    n = 300
    rng = np.random.default_rng(3)
    p = (rng.normal(scale=0.2, size=M.NPARAMS)).astype(np.float32)
    X, T = data(4, n)
    m = model_with(sv, p)
    try:
        sv.sv_cost_model_train(m, X, T, epochs=1, batch=n, lr=1e-2, seed=5)
        p1 = sv.sv_cost_model_get_params(m)
    finally:
        sv.sv_cost_model_destroy(m)
    p64 = p.astype(np.float64)
    g = M.gradient(p64, X.astype(np.float64), T.astype(np.float64))
    want, _, _ = M.adam_step(p64, np.zeros_like(g), np.zeros_like(g), g, 1, lr=1e-2)
    # a first Adam step moves each coordinate by lr * g / (|g| + eps): where
    # |g| is tiny the FP32 gradient's sign decides, so compare the rest
    big = np.abs(g) > 1e-5
    assert np.max(np.abs(p1[big] - want[big])) <= 1e-5


def test_training_reduces_loss_and_generalises(sv):
    """A smooth target of the features is learnt: held-out MSE far below the
    variance of the target."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 1, size=(12000, M.NF)).astype(np.float32)
    w = rng.normal(size=M.NF)
    T = (np.sin(X @ w) + 0.5 * X[:, 3] * X[:, 40]).astype(np.float32)
    m = sv.sv_cost_model_create(11)
    try:
        losses = sv.sv_cost_model_train(m, X[:10000], T[:10000], epochs=60, batch=512, lr=2e-3,
                                        seed=1)
        pred = sv.sv_cost_model_predict(m, X[10000:])
    finally:
        sv.sv_cost_model_destroy(m)
    assert losses[-1] < 0.2 * losses[0]
    assert np.mean((pred - T[10000:]) ** 2) < 0.1 * np.var(T[10000:])


def test_save_load_round_trip(sv, tmp_path):
    m = sv.sv_cost_model_create(123)
    try:
        p = sv.sv_cost_model_get_params(m)
        path = str(tmp_path / "m.svcm")
        sv.sv_cost_model_save(m, path)
    finally:
        sv.sv_cost_model_destroy(m)
    m2 = sv.sv_cost_model_load(path)
    try:
        assert np.array_equal(sv.sv_cost_model_get_params(m2), p)
    finally:
        sv.sv_cost_model_destroy(m2)
