"""FP64 oracle of the planner's cost model (a small MLP), in NumPy.

TEST INFRASTRUCTURE ONLY: the test-suite may import this module; the library
does not.  It shares no code with the CUDA kernels that train and evaluate
the same network on the GPU.

The network: x (NF inputs) -> Linear(64) -> ReLU -> Linear(64) -> ReLU ->
Linear(1), trained on the mean squared error with Adam.  Its parameters are
one flat vector, in this order (row-major):
    W1 [NF][64], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]
so that z1_j = b1_j + sum_i x_i W1[i][j], and likewise for the other layers.
ReLU'(z) is taken as 1 for z > 0 and 0 otherwise.

Adam (Kingma and Ba, "Adam: A Method for Stochastic Optimization", 2015,
Algorithm 1): m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
m_hat = m / (1 - b1^t);  v_hat = v / (1 - b2^t);
theta <- theta - lr * m_hat / (sqrt(v_hat) + eps).
"""
from __future__ import annotations

import numpy as np

NF = 52
H = 64
NPARAMS = NF * H + H + H * H + H + H + 1


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    assert p.size == NPARAMS
    o = 0
    W1 = p[o:o + NF * H].reshape(NF, H); o += NF * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, [b3]]).astype(np.float64)


def forward(p: np.ndarray, X: np.ndarray):
    """Outputs y (N,) and the intermediate activations."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    h1 = np.where(z1 > 0, z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.where(z2 > 0, z2, 0.0)
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2)


def loss(p: np.ndarray, X: np.ndarray, T: np.ndarray) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(p: np.ndarray, X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """d loss / d p by the chain rule, layer by layer from the output."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    n = y.size
    dy = 2.0 * (y - np.asarray(T, dtype=np.float64)) / n        # dL/dy
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)                            # dL/dz2
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)                                # dL/dz1
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def finite_difference(p: np.ndarray, X: np.ndarray, T: np.ndarray, idx, h: float = 1e-6):
    """Central differences (L(p + h e_i) - L(p - h e_i)) / 2h for each i in idx."""
    p = np.asarray(p, dtype=np.float64)
    out = []
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        out.append((loss(p + e, X, T) - loss(p - e, X, T)) / (2 * h))
    return np.array(out)


def adam_step(p, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step t >= 1); returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
