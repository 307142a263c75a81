"""Batched replicas: many independent lattices advanced in one persistent launch.

The batched-replica workload: n replicas with L drawn uniformly from {64, 128, 256, 512,
1024}, r uniform in [3.5, 4.2], K = 0.5, independent seeds, Bernoulli(1/2) starts (Section
III), n_mcs MCS each; the batch autotuner picks the CTA size and warps per replica, the
persistent launch is captured in a CUDA graph. For comparison the same replicas are also
advanced with one launch sequence per replica through the single-lattice path: all of them for
the same number of MCS (--compare-all, measured), or a sample whose rate is scaled to the
workload.

    python -m paper_1704_08098_gb300.replicas --n 512 --mcs 5000
    python -m paper_1704_08098_gb300.replicas --n 512 --mcs 200 --compare-all
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs


def make_workload(n: int, seed: int = 7):
    L = inputs.replica_sizes(n, (64, 128, 256, 512, 1024), seed)
    r = inputs.uniform_params(n, 3.5, 4.2, seed + 1)
    seeds = np.arange(1000, 1000 + n, dtype=np.uint64)
    return L.astype(np.int32), r, seeds


def run(n: int = 512, n_mcs: int = 5000, chunk: int = 500, tune_mcs: int = 20,
        per_replica_sample: int = 16, per_replica_mcs: int = 50, seed: int = 7,
        autotune: bool = True, compare: bool = True) -> dict:
    import torch
    from . import build, pgg
    build.build()
    L, r, seeds = make_workload(n, seed)
    stream = torch.cuda.current_stream()
    sites_per_mcs = float(np.sum(L.astype(np.float64) ** 2))
    out = {"n": n, "n_mcs": n_mcs, "sizes": {int(x): int((L == x).sum()) for x in np.unique(L)}}
    with pgg.Batch(L, r, 0.5, seeds, stream=stream.cuda_stream) as b:
        b.seed(0.5)
        out["autotune"] = b.autotune(tune_mcs) if autotune else None
        torch.cuda.synchronize()
        counts = np.zeros((n, n_mcs), dtype=np.uint32)
        dev = torch.zeros((n, chunk), dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gpu_ms = 0.0
        done = 0
        t0 = time.perf_counter()
        while done < n_mcs:
            m = min(chunk, n_mcs - done)
            e0.record(stream)
            b.step_mcs(m, dev.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            gpu_ms += e0.elapsed_time(e1)
            counts[:, done:done + m] = dev.view(-1)[: n * m].cpu().numpy().view(np.uint32).reshape(n, m)
            done += m
        wall = time.perf_counter() - t0
    out["batched"] = {"gpu_s": gpu_ms / 1e3, "wall_s": wall,
                      "site_updates_per_s": sites_per_mcs * n_mcs / (gpu_ms / 1e3)}
    out["final_rho"] = {"mean": float((counts[:, -1] / L.astype(np.float64) ** 2).mean()),
                        "absorbed": int((counts[:, -1] == 0).sum())}
    if not compare:
        return out
    # one launch sequence per replica (the single-lattice API): every replica when
    # per_replica_sample >= n (a measured comparison over the same MCS), else a sample of them
    # whose rate is scaled to the workload
    full = per_replica_sample >= n
    idx = np.arange(n) if full else np.random.default_rng(seed).choice(n, size=per_replica_sample, replace=False)
    mcs = n_mcs if full else per_replica_mcs
    per_ms = 0.0
    sample_sites = 0.0
    per_counts_match = True
    for i in idx:
        with pgg.Lattice(int(L[i]), float(r[i]), 0.5, layout="bitpack", stream=stream.cuda_stream) as lat:
            lat.seed(int(seeds[i]), 0.5)
            if not full:
                lat.advance(2)
            torch.cuda.synchronize()
            e0.record(stream)
            lat.advance(mcs)
            e1.record(stream)
            torch.cuda.synchronize()
            per_ms += e0.elapsed_time(e1)
            sample_sites += float(L[i]) ** 2 * mcs
            if full:
                per_counts_match &= lat.count() == int(counts[i, -1])
    rate = sample_sites / (per_ms / 1e3)
    if full:
        out["per_replica"] = {"gpu_s": per_ms / 1e3, "site_updates_per_s": rate, "replicas": int(n), "mcs": mcs,
                              "measured": True, "final_counts_equal_batched": bool(per_counts_match)}
        out["speedup"] = out["per_replica"]["gpu_s"] / out["batched"]["gpu_s"]
    else:
        out["per_replica"] = {"site_updates_per_s": rate, "sample_replicas": int(len(idx)),
                              "sample_mcs": per_replica_mcs, "measured": False,
                              "est_gpu_s_for_workload": sites_per_mcs * n_mcs / rate}
        out["speedup"] = out["per_replica"]["est_gpu_s_for_workload"] / out["batched"]["gpu_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--mcs", type=int, default=5000)
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--no-autotune", action="store_true", help="library default CTA size and team warps")
    ap.add_argument("--no-compare", action="store_true", help="skip the one-launch-sequence-per-replica timing")
    ap.add_argument("--compare-all", action="store_true",
                    help="run every replica through the single-lattice path for the same MCS (measured, "
                         "not extrapolated from a sample)")
    args = ap.parse_args()
    print(json.dumps(run(args.n, args.mcs, args.chunk, autotune=not args.no_autotune,
                         compare=not args.no_compare,
                         per_replica_sample=args.n if args.compare_all else 16)))


if __name__ == "__main__":
    main()
