"""Bisection for the absorbing transition r_c, plain or gated by the learned surrogate.

Section V locates the C+D -> D transition at r_c = 3.7443(4) for K = 0.5 (Fig. 4): below r_c
every run ends in the absorbing all-defector state, above it cooperators survive. A probe at
synergy factor r runs `replicas` independent lattices; it is "absorbing" when the majority
reached rho_C = 0 within T_max MCS (absorption is exact and final, so a probe stops as soon
as a majority is absorbed). Bisection on [lo, hi] shrinks the bracket to `width`. A finite
T_max places the transition slightly below r_c: runs just below it need longer to die.

With a surrogate, each probe first runs FEATURE_MCS = 200 MCS, asks the network for
P(absorbing) of every replica, and decides at once when the mean is beyond `conf` (or below
1 - conf); otherwise it falls back to the full simulation, which stays the judge. GPU time is
the sum of CUDA-event times of every simulation and inference call.

    python -m paper_1704_08098_gb300.rc_search --L 1024 --surrogate surrogate.npz
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from .surrogate import FEATURE_MCS, Surrogate


class GpuTimer:
    def __init__(self):
        import torch
        self.torch = torch
        self.ms = 0.0

    def __enter__(self):
        t = self.torch
        self.s = t.cuda.current_stream()
        self.e0, self.e1 = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        self.e0.record(self.s)
        return self

    def __exit__(self, *exc):
        self.e1.record(self.s)
        self.torch.cuda.synchronize()
        self.ms += self.e0.elapsed_time(self.e1)


def probe(r: float, L: int, T_max: int, replicas: int, seed: int, surrogate=None,
          conf: float = 0.99, chunk: int = 500, timer: GpuTimer | None = None) -> dict:
    import torch
    from . import pgg
    seeds = np.arange(seed, seed + replicas, dtype=np.uint64)
    N = float(L * L)
    dev = torch.zeros(replicas * max(chunk, FEATURE_MCS), dtype=torch.int32, device="cuda")
    timer = timer or GpuTimer()
    out = {"r": r, "mcs": 0, "decided_by": "simulation"}
    with pgg.Batch(np.full(replicas, L, np.int32), np.full(replicas, r), 0.5, seeds,
                   stream=torch.cuda.current_stream().cuda_stream) as b:
        with timer:
            b.seed(0.5)
            b.step_mcs(FEATURE_MCS, dev.data_ptr())
        prefix = dev[: replicas * FEATURE_MCS].cpu().numpy().view(np.uint32).reshape(replicas, FEATURE_MCS)
        out["mcs"] = FEATURE_MCS
        absorbed = prefix[:, -1] == 0
        if surrogate is not None:
            with timer:
                p, _ = surrogate.predict(prefix / N, r, 0.5)
            out["p_mean"] = float(p.mean())
            if p.mean() > conf or p.mean() < 1 - conf:
                out["decided_by"] = "surrogate"
                out["absorbing"] = bool(p.mean() > 0.5)
                return out
        done = FEATURE_MCS
        while done < T_max and absorbed.sum() * 2 <= replicas:
            m = min(chunk, T_max - done)
            with timer:
                b.step_mcs(m, dev.data_ptr())
            c = dev[: replicas * m].cpu().numpy().view(np.uint32).reshape(replicas, m)
            absorbed |= (c == 0).any(axis=1)
            done += m
        out["mcs"] = done
        out["absorbed"] = int(absorbed.sum())
        out["absorbing"] = bool(absorbed.sum() * 2 > replicas)
    return out


def bisect(L: int = 1024, lo: float = 3.5, hi: float = 4.2, width: float = 0.01,
           T_max: int = 50000, replicas: int = 16, surrogate=None, conf: float = 0.99,
           seed: int = 500, judge: bool = False) -> dict:
    timer = GpuTimer()
    probes = []
    k = 0
    while hi - lo > width:
        r = 0.5 * (lo + hi)
        pr = probe(r, L, T_max, replicas, seed + 1000 * k, surrogate, conf, timer=timer)
        if judge and pr["decided_by"] == "surrogate":
            # the full simulation (same seeds), outside the timed search, judges the decision
            full = probe(r, L, T_max, replicas, seed + 1000 * k)
            pr["judge_absorbing"] = full["absorbing"]
            pr["judge_agrees"] = full["absorbing"] == pr["absorbing"]
        probes.append(pr)
        if pr["absorbing"]:
            lo = r  # cooperators die out: r_c lies above r
        else:
            hi = r
        k += 1
    return {"bracket": [lo, hi], "center": 0.5 * (lo + hi), "gpu_ms": timer.ms, "probes": probes}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=1024)
    ap.add_argument("--T", type=int, default=50000)
    ap.add_argument("--replicas", type=int, default=16)
    ap.add_argument("--judge", action="store_true", help="re-run surrogate decisions in full")
    ap.add_argument("--width", type=float, default=0.01)
    ap.add_argument("--surrogate", default=None)
    ap.add_argument("--conf", type=float, default=0.99)
    ap.add_argument("--plain", action="store_true", help="also run the plain bisection")
    args = ap.parse_args()
    res = {}
    if args.surrogate:
        params = np.load(args.surrogate)["params"]
        s = Surrogate(params)
        res["surrogate"] = bisect(args.L, T_max=args.T, replicas=args.replicas, width=args.width,
                                  surrogate=s, conf=args.conf, judge=args.judge)
        s.close()
    if args.plain or not args.surrogate:
        res["plain"] = bisect(args.L, T_max=args.T, replicas=args.replicas, width=args.width)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
