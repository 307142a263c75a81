"""FP64 oracle of the surrogate MLP (test infrastructure only).

The surrogate reads the first 200 samples of the cooperator fraction rho_C(t) (Eq. (4)) of a
run plus its (r, K) and predicts P(absorbing) and the stationary rho_C. Architecture:
x (202) -> relu(W1 x + b1) (128) -> relu(W2 h1 + b2) (128) -> z = W3 h2 + b3 (2);
p = sigmoid(z_0), rho = sigmoid(z_1). The GPU evaluates it with BF16 parameters and FP32
accumulation; this oracle evaluates the same BF16-rounded parameters in float64.

Loss (per batch of B samples with labels y_abs in {0, 1}, y_rho in [0, 1], mask in {0, 1}):
    L = (1/B) sum_b [ -y_abs log p - (1 - y_abs) log(1 - p) ] + (1/B) sum_b mask (rho - y_rho)^2
Adam (Kingma & Ba, ICLR 2015) with bias correction updates the FP32 master parameters.

Pins (tests/test_mlp_oracle.py): analytic gradients against central finite differences,
closed forms (zero weights), BF16 round-to-nearest-even on hand-picked values, Adam against
its update written out for one step.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 202, 128, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest, ties to even) -> float64 (exact)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((u >> 16) & 1)
    r = ((u + rounding) >> 16) << 16
    # NaN inputs are not expected; keep them NaN
    r = np.where((u & 0x7FFFFFFF) > 0x7F800000, u | 0x00400000, r)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta_bf16: np.ndarray, X: np.ndarray):
    """Forward pass in float64 with the given (already BF16-rounded) parameters."""
    P = unpack(np.asarray(theta_bf16, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["W3"].T + P["b3"]
    return dict(a1=a1, h1=h1, a2=a2, h2=h2, z=z, p=sigmoid(z[:, 0]), rho=sigmoid(z[:, 1]))


def loss(theta_bf16: np.ndarray, X: np.ndarray, Y: np.ndarray) -> float:
    f = forward(theta_bf16, X)
    B = X.shape[0]
    y, yr, m = Y[:, 0], Y[:, 1], Y[:, 2]
    bce = -(y * np.log(f["p"]) + (1 - y) * np.log(1 - f["p"]))
    mse = m * (f["rho"] - yr) ** 2
    return float((bce.sum() + mse.sum()) / B)


def gradients(theta_bf16: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Analytic gradient of loss() with respect to the parameters (back-propagation)."""
    P = unpack(np.asarray(theta_bf16, dtype=np.float64))
    f = forward(theta_bf16, X)
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    y, yr, m = Y[:, 0], Y[:, 1], Y[:, 2]
    dz = np.zeros_like(f["z"])
    dz[:, 0] = (f["p"] - y) / B                                           # BCE through sigmoid
    dz[:, 1] = m * 2.0 * (f["rho"] - yr) * f["rho"] * (1 - f["rho"]) / B  # MSE through sigmoid
    g = {}
    g["W3"] = dz.T @ f["h2"]
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ P["W3"]
    da2 = dh2 * (f["a2"] > 0)
    g["W2"] = da2.T @ f["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * (f["a1"] > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1) in float64; returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
