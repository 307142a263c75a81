"""The learned surrogate for the r_c search: data generation, training, inference.

Data: n runs of the game on an L x L lattice (default L = 256) with r uniform in [3.5, 4.2],
K = 0.5, Bernoulli(1/2) starts (Section III), advanced by the batched simulator. Features are
the first 200 values of rho_C(t) (Eq. (4)) plus the normalised (r, K); labels are whether
the run reached the absorbing all-defector state within T_label MCS (absorption is exact and
final: no rule creates a cooperator from none) and, for runs still active, the mean rho_C
over the last `window` MCS (the stationary density of Section III).

Training runs entirely in the library's CUDA kernels (pgg_mlp_train_step); this module only
shuffles indices and moves batches.

    python -m paper_1704_08098_gb300.surrogate --n 20000 --out surrogate.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs

FEATURE_MCS = 200
R_CENTER, R_SCALE = 3.85, 0.35
K_CENTER, K_SCALE = 0.5, 0.5


def features(rho_prefix: np.ndarray, r, K) -> np.ndarray:
    """Rows [rho(1) .. rho(200), (r - 3.85) / 0.35, (K - 0.5) / 0.5] as float32."""
    rho_prefix = np.asarray(rho_prefix, dtype=np.float32)
    n = rho_prefix.shape[0]
    r = np.broadcast_to(np.asarray(r, dtype=np.float64), (n,))
    K = np.broadcast_to(np.asarray(K, dtype=np.float64), (n,))
    X = np.empty((n, FEATURE_MCS + 2), dtype=np.float32)
    X[:, :FEATURE_MCS] = rho_prefix[:, :FEATURE_MCS]
    X[:, FEATURE_MCS] = ((r - R_CENTER) / R_SCALE).astype(np.float32)
    X[:, FEATURE_MCS + 1] = ((K - K_CENTER) / K_SCALE).astype(np.float32)
    return X


def generate(n: int = 20000, L: int = 256, T_label: int = 5000, window: int = 1000,
             chunk: int = 500, seed: int = 11, r_lo: float = 3.5, r_hi: float = 4.2):
    """Simulate n runs with the batched engine; returns (X, Y, meta)."""
    import torch
    from . import build, pgg
    build.build()
    assert T_label >= FEATURE_MCS and window <= T_label
    r = inputs.uniform_params(n, r_lo, r_hi, seed)
    seeds = np.arange(10_000_000 + seed * 100_000, 10_000_000 + seed * 100_000 + n, dtype=np.uint64)
    Ls = np.full(n, L, dtype=np.int32)
    stream = torch.cuda.current_stream()
    dev = torch.zeros(n * max(chunk, FEATURE_MCS), dtype=torch.int32, device="cuda")
    N = float(L * L)
    t0 = time.perf_counter()
    with pgg.Batch(Ls, r, 0.5, seeds, stream=stream.cuda_stream) as b:
        b.seed(0.5)
        b.step_mcs(FEATURE_MCS, dev.data_ptr())
        torch.cuda.synchronize()
        prefix = dev[: n * FEATURE_MCS].cpu().numpy().view(np.uint32).reshape(n, FEATURE_MCS) / N
        absorbed = prefix[:, -1] == 0
        tail_sum = np.zeros(n)
        done = FEATURE_MCS
        while done < T_label:
            m = min(chunk, T_label - done)
            b.step_mcs(m, dev.data_ptr())
            torch.cuda.synchronize()
            c = dev[: n * m].cpu().numpy().view(np.uint32).reshape(n, m) / N
            absorbed |= (c == 0).any(axis=1)
            lo = max(done, T_label - window)
            if done + m > lo:
                tail_sum += c[:, lo - done:].sum(axis=1)
            done += m
    gen_s = time.perf_counter() - t0
    y = absorbed.astype(np.float32)
    rho = np.where(absorbed, 0.0, tail_sum / window).astype(np.float32)
    Y = np.stack([y, rho, 1.0 - y], axis=1).astype(np.float32)
    X = features(prefix, r, 0.5)
    meta = {"n": n, "L": L, "T_label": T_label, "window": window, "absorbed_frac": float(y.mean()),
            "seconds": gen_s, "r": r}
    return X, Y, meta


def train(X: np.ndarray, Y: np.ndarray, epochs: int = 40, batch: int = 256, lr: float = 1e-3,
          seed: int = 5, init=None):
    """Adam on the GPU through pgg_mlp_train_step; returns (master params, loss per epoch)."""
    import torch
    from . import build, pgg
    build.build()
    n = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    rng = np.random.default_rng(seed)
    history = []
    loss = torch.zeros(1, device="cuda")
    with pgg.MLP(batch) as net:
        net.set_params(inputs.mlp_init_params(seed) if init is None else init)
        xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device="cuda")
        yb = torch.empty((batch, 3), dtype=torch.float32, device="cuda")
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).cuda()
            tot, steps = 0.0, 0
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                torch.index_select(Xd, 0, idx, out=xb)
                torch.index_select(Yd, 0, idx, out=yb)
                net.train_step(xb.data_ptr(), yb.data_ptr(), batch, lr, loss.data_ptr())
                tot += float(loss.item()) if steps % 16 == 0 else 0.0
                steps += 1
            history.append(tot / max(1, (steps + 15) // 16))
        master, _ = net.get_params()
    return master, history


class Surrogate:
    """Inference with trained parameters (pgg_mlp_forward on the GPU)."""

    def __init__(self, params: np.ndarray, max_batch: int = 4096):
        from . import build, pgg
        build.build()
        self.net = pgg.MLP(max_batch)
        self.net.set_params(params)
        self.max_batch = max_batch

    def predict(self, rho_prefix: np.ndarray, r, K) -> tuple[np.ndarray, np.ndarray]:
        import torch
        X = features(rho_prefix, r, K)
        Xd = torch.from_numpy(X).cuda()
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
        for s in range(0, X.shape[0], self.max_batch):
            B = min(self.max_batch, X.shape[0] - s)
            self.net.forward(Xd[s:].data_ptr(), B, out[s:].data_ptr())
        o = out.cpu().numpy()
        return o[:, 0], o[:, 1]

    def close(self):
        self.net.close()


def evaluate(params: np.ndarray, X: np.ndarray, Y: np.ndarray, conf: float = 0.95) -> dict:
    """Accuracy of the absorbing classifier and the density error on held-out rows."""
    import torch
    from . import build, pgg
    build.build()
    with pgg.MLP(max(1, X.shape[0])) as net:
        net.set_params(params)
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
        net.forward(Xd.data_ptr(), X.shape[0], out.data_ptr())
        o = out.cpu().numpy()
    p, rho = o[:, 0], o[:, 1]
    y = Y[:, 0] > 0.5
    sure = (p > conf) | (p < 1 - conf)
    active = ~y
    return {"accuracy": float(((p > 0.5) == y).mean()), "confident_frac": float(sure.mean()),
            "confident_accuracy": float(((p[sure] > 0.5) == y[sure]).mean()) if sure.any() else None,
            "rho_mae_active": float(np.abs(rho[active] - Y[active, 1]).mean()) if active.any() else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--T", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default="surrogate.npz")
    args = ap.parse_args()
    X, Y, meta = generate(args.n, args.L, args.T)
    n_train = int(0.9 * len(X))
    params, hist = train(X[:n_train], Y[:n_train], epochs=args.epochs)
    ev = evaluate(params, X[n_train:], Y[n_train:])
    np.savez(args.out, params=params, loss=np.asarray(hist))
    meta.pop("r")
    print(json.dumps({"data": meta, "loss_first": hist[0], "loss_last": hist[-1], "heldout": ev}))


if __name__ == "__main__":
    main()
