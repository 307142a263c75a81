"""The FP64 surrogate-network oracle against finite differences and closed forms (CPU)."""
import numpy as np

from oracle import mlp as M
from paper_1704_08098_gb300 import inputs


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = inputs.mlp_init_params(3).astype(np.float64) + rng.normal(0, 0.01, M.N_PARAMS)
    X = inputs.random_features(6, 4).astype(np.float64)
    Y = inputs.random_labels(6, 5).astype(np.float64)
    g = M.gradients(theta, X, Y)
    idx = np.concatenate([rng.choice(M.N_PARAMS, 60, replace=False),
                          np.arange(M.N_PARAMS - 258, M.N_PARAMS)])  # W3, b3 in full
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss(tp, X, Y) - M.loss(tm, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_weights_closed_form():
    theta = np.zeros(M.N_PARAMS)
    X = inputs.random_features(5, 1).astype(np.float64)
    Y = inputs.random_labels(5, 2).astype(np.float64)
    f = M.forward(theta, X)
    assert np.allclose(f["p"], 0.5) and np.allclose(f["rho"], 0.5)
    want = np.log(2.0) + np.mean(Y[:, 2] * (0.5 - Y[:, 1]) ** 2)
    assert abs(M.loss(theta, X, Y) - want) < 1e-15


def test_bf16_round_to_nearest_even():
    one = 1.0
    cases = {one: one, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6,
             1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7, -2.5: -2.5, 3.0e-3: 0.0030059814453125}
    for x, want in cases.items():
        assert M.bf16_round(np.array([x], np.float32))[0] == want, x


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t1, m, v = M.adam_step(theta, np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # bias-corrected first moments equal g and second moments g^2: a step of lr * sign(g)
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
