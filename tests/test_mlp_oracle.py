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


def test_forward_hand_worked_sparse_network():
    """A network with a handful of non-zero weights (all exact in BF16), worked by hand: the
    first layer multiplies x by W1 (output unit i reads input j through W1[i, j]) and adds b1,
    the ReLUs cut negative and zero pre-activations, and the sigmoids of z give p and rho."""
    P = {name: np.zeros(shape) for name, shape in M.SHAPES}
    P["W1"][0, 0], P["W1"][0, 1], P["b1"][0] = 2.0, 1.0, 0.25
    P["W1"][1, 0], P["b1"][1] = -1.0, 0.125
    P["W1"][2, 200], P["b1"][2] = 1.0, -3.5
    P["W2"][0, 0], P["W2"][0, 2] = 4.0, -1.0
    P["W2"][1, 1], P["W2"][1, 2], P["b2"][1] = 100.0, 2.0, -2.0
    P["W2"][5, 0], P["b2"][5] = -8.0, 3.0
    P["W3"][0, 0], P["W3"][0, 5], P["b3"][0] = 2.0, -3.0, 0.5
    P["W3"][1, 5] = 0.75
    theta = np.concatenate([P[name].reshape(-1) for name, _ in M.SHAPES])
    assert np.array_equal(M.bf16_round(theta.astype(np.float32)), theta)
    X = np.zeros((2, M.N_IN))
    X[0, 0], X[0, 1], X[0, 200], X[0, 201] = 0.5, -1.0, 4.0, 0.5
    X[1, 0], X[1, 200], X[1, 201] = 1.0, 3.5, 0.5
    f = M.forward(theta, X)
    # row 0: a1 = (0.25, -0.375, 0.5) -> h1 = (0.25, 0, 0.5); h2_0 = 1 - 0.5, h2_1 = relu(1 - 2) = 0,
    # h2_5 = -2 + 3; z = (1 - 3 + 0.5, 0.75)
    # row 1: h1 = (2.25, 0, relu(0) = 0); h2_0 = 9, h2_5 = relu(-15) = 0; z = (18.5, 0)
    assert np.allclose(f["h1"][:, :3], [[0.25, 0.0, 0.5], [2.25, 0.0, 0.0]], rtol=0, atol=1e-15)
    assert np.allclose(f["z"], [[-1.5, 0.75], [18.5, 0.0]], rtol=0, atol=1e-15)
    want_p = np.array([1.0 / (1.0 + np.exp(1.5)), 1.0 / (1.0 + np.exp(-18.5))])
    want_rho = np.array([1.0 / (1.0 + np.exp(-0.75)), 0.5])
    assert np.allclose(f["p"], want_p, rtol=1e-15, atol=0) and np.allclose(f["rho"], want_rho, rtol=1e-15, atol=0)
    assert abs(f["p"][0] - 0.18242552380635635) < 1e-15 and abs(f["rho"][0] - 0.679178699175393) < 1e-15
    # loss: labels (absorbed, rho, mask) = (1, 0.6, 1) and (0, 0.2, 0)
    Y = np.array([[1.0, 0.6, 1.0], [0.0, 0.2, 0.0]])
    want = (-np.log(want_p[0]) - np.log(1.0 - want_p[1]) + (want_rho[0] - 0.6) ** 2) / 2.0
    assert abs(M.loss(theta, X, Y) - want) < 1e-14
