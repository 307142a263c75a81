"""Stationary cooperator density and long-run throughput at L = 4096 (Section III, Eq. (4)).

Runs the game from Bernoulli(1/2) starts at K = 0.5 for r in {3.5, 3.7, 3.9, 4.5, 5.0}, seed
1..5 (one per r), for 20000 MCS in both lattice layouts, and reports the mean rho_C over the
last 5000 MCS (the relaxation before is discarded, as Section III prescribes). Both layouts
run the same random stream, so their per-MCS counts must agree exactly; the driver checks
that. With --long it also times the paper's own throughput workload, 10^6 MCS at L = 4096,
r = 3.98 (Section V), on the bit-packed lattice.

    python -m paper_1704_08098_gb300.stationary --L 4096 --T 20000 --window 5000 --long 1000000
"""
from __future__ import annotations

import argparse
import json

import numpy as np

R_VALUES = (3.5, 3.7, 3.9, 4.5, 5.0)


def run_one(L: int, r: float, K: float, seed: int, T: int, window: int, layout: str,
            chunk: int = 1000) -> dict:
    import torch
    from . import pgg
    stream = torch.cuda.current_stream()
    counts = torch.zeros(chunk, dtype=torch.int64, device="cuda")
    per_mcs = np.empty(T, dtype=np.uint64)
    with pgg.Lattice(L, r, K, layout=layout, stream=stream.cuda_stream) as lat:
        lat.seed(seed, 0.5)
        if L >= 1024:
            lat.autotune(2)  # untimed; restores the lattice and step counter
        sched = lat.schedule()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gpu_ms = 0.0
        done = 0
        while done < T:
            m = min(chunk, T - done)
            e0.record(stream)
            lat.step_mcs(m, counts.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            gpu_ms += e0.elapsed_time(e1)
            per_mcs[done:done + m] = counts[:m].cpu().numpy().view(np.uint64)
            done += m
    N = float(L) * L
    rho = per_mcs.astype(np.float64) / N
    return {"layout": layout, "r": r, "seed": seed, "rho_stationary": float(rho[T - window:].mean()),
            "rho_std_window": float(rho[T - window:].std()), "rho_T": float(rho[-1]),
            "absorbed": bool(per_mcs[-1] == 0), "gpu_s": gpu_ms / 1e3,
            "site_updates_per_s": N * T / (gpu_ms / 1e3), "schedule": sched,
            "counts_digest": int(np.bitwise_xor.reduce(per_mcs * np.arange(1, T + 1, dtype=np.uint64)))}


def long_run(L: int, r: float, K: float, T: int, seed: int = 1, layout: str = "bitpack",
             chunk: int = 10000) -> dict:
    import torch
    from . import pgg
    stream = torch.cuda.current_stream()
    with pgg.Lattice(L, r, K, layout=layout, stream=stream.cuda_stream) as lat:
        lat.seed(seed, 0.5)
        if L >= 1024:
            lat.autotune(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        done = 0
        while done < T:
            m = min(chunk, T - done)
            lat.advance(m)
            done += m
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        rho = lat.count() / float(L * L)
        sched = lat.schedule()
    return {"L": L, "r": r, "K": K, "mcs": T, "layout": layout, "gpu_s": s,
            "site_updates_per_s": float(L) * L * T / s, "rho_T": rho, "schedule": sched,
            "paper_gpu_s_bound": 5400.0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--T", type=int, default=20000)
    ap.add_argument("--window", type=int, default=5000)
    ap.add_argument("--long", type=int, default=0, help="MCS of the r = 3.98 throughput run (0: skip)")
    args = ap.parse_args()
    from . import build
    build.build()
    runs = []
    for layout in ("bitpack", "u8"):
        for i, r in enumerate(R_VALUES):
            runs.append(run_one(args.L, r, 0.5, i + 1, args.T, args.window, layout))
    agree = all(a["counts_digest"] == b["counts_digest"]
                for a, b in zip(runs[:len(R_VALUES)], runs[len(R_VALUES):]))
    out = {"L": args.L, "K": 0.5, "T": args.T, "window": args.window, "runs": runs,
           "layouts_agree_exactly": agree}
    if args.long:
        out["long"] = long_run(args.L, 3.98, 0.5, args.long)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
