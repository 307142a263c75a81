"""The surrogate network's CUDA kernels against the FP64 oracle (same BF16 parameters)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1704_08098_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1704_08098_gb300 import build, pgg
    build.build()
    return torch, pgg


def params(seed, noise=0.05):
    rng = np.random.default_rng(seed)
    p = inputs.mlp_init_params(seed)
    return (p + rng.normal(0, noise, p.size)).astype(np.float32)


@pytest.mark.parametrize("B", [1, 37, 256, 1000])
def test_forward_matches_fp64(env, B):
    torch, pgg = env
    theta = params(1)
    X = inputs.random_features(B, 2)
    with pgg.MLP(1024) as net:
        net.set_params(theta)
        _, q = net.get_params()
        assert np.array_equal(q.astype(np.float64), M.bf16_round(theta))
        Xd = torch.from_numpy(X).cuda()
        out = torch.empty((B, 2), dtype=torch.float32, device="cuda")
        net.forward(Xd.data_ptr(), B, out.data_ptr())
        got = out.cpu().numpy().astype(np.float64)
    f = M.forward(M.bf16_round(theta), X)
    want = np.stack([f["p"], f["rho"]], axis=1)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want)), np.max(np.abs(got - want) / np.abs(want))


def test_loss_and_gradient_match_fp64(env):
    torch, pgg = env
    theta = params(3)
    B = 128
    X, Y = inputs.random_features(B, 4), inputs.random_labels(B, 5)
    with pgg.MLP(B) as net:
        net.set_params(theta)
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(M.N_PARAMS, device="cuda")
        net.loss_grad(Xd.data_ptr(), Yd.data_ptr(), B, loss.data_ptr(), grad.data_ptr())
        g = grad.cpu().numpy().astype(np.float64)
        lo = float(loss.item())
    tq = M.bf16_round(theta)
    assert abs(lo - M.loss(tq, X, Y)) <= 1e-5 * abs(M.loss(tq, X, Y))
    want = M.gradients(tq, X, Y)
    scale = np.abs(want).max()
    assert np.all(np.abs(g - want) <= 1e-4 * np.abs(want) + 1e-5 * scale)


def test_adam_steps_match_fp64_and_are_deterministic(env):
    torch, pgg = env
    theta = params(7)
    B = 64
    X, Y = inputs.random_features(B, 8), inputs.random_labels(B, 9)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    runs = []
    for _ in range(2):
        with pgg.MLP(B) as net:
            net.set_params(theta)
            for _ in range(3):
                net.train_step(Xd.data_ptr(), Yd.data_ptr(), B, 1e-3)
            runs.append(net.get_params()[0])
    assert np.array_equal(runs[0], runs[1])
    th, m, v = theta.astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    for t in (1, 2, 3):
        g = M.gradients(M.bf16_round(th.astype(np.float32)), X, Y)
        th, m, v = M.adam_step(th, m, v, g, t, lr=1e-3)
    # each Adam step moves a parameter by at most lr; FP32 vs FP64 differences stay far below
    assert np.max(np.abs(runs[0] - th)) < 1e-5


def test_training_reduces_loss(env):
    torch, pgg = env
    rng = np.random.default_rng(0)
    B = 256
    X = inputs.random_features(B, 11)
    y = (X[:, :200].mean(axis=1) < 0.5).astype(np.float32)   # a learnable rule
    Y = np.stack([y, np.where(y > 0, 0, X[:, :200].mean(axis=1)), 1 - y], axis=1).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    loss = torch.zeros(1, device="cuda")
    with pgg.MLP(B) as net:
        net.set_params(inputs.mlp_init_params(12))
        net.loss_grad(Xd.data_ptr(), Yd.data_ptr(), B, loss.data_ptr(), None)
        first = float(loss.item())
        for _ in range(300):
            net.train_step(Xd.data_ptr(), Yd.data_ptr(), B, 3e-3, loss.data_ptr())
        net.loss_grad(Xd.data_ptr(), Yd.data_ptr(), B, loss.data_ptr(), None)
        last = float(loss.item())
    assert last < 0.5 * first
