"""Critical decay of the cooperator fraction near the absorbing transition (Section V).

The transition belongs to the directed-percolation class (Section V, Eq. (5)): below r_c every
run ends absorbed, above it the stationary cooperator fraction scales as (r - r_c)^beta. This
driver runs one lattice per r on its own CUDA stream (so all r advance concurrently on the
GPU) from Bernoulli(1/2) starts, records rho_C at log-spaced times t = floor(10^(m/20)), and
reports per r the late-time log-log slope and the late-time density, with a fit of the
late-time densities to A (r - r_c)^beta. From a random start rho_C first collapses and then
recovers above r_c, so near r_c the late-time density is stationary only for times far
beyond the critical relaxation time; the fit is as good as the run is long.

    python -m paper_1704_08098_gb300.critical --L 8192 --T 100000
    python -m paper_1704_08098_gb300.critical --L 4096 --T 100000 --r-lo 3.75 --r-hi 3.90 --r-step 0.01
    python -m paper_1704_08098_gb300.critical --anneal --L 2048 --T 100000 --r-lo 3.748 --r-hi 3.800 --r-step 0.004
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def log_times(T: int) -> np.ndarray:
    t = np.unique(np.floor(10.0 ** (np.arange(0, int(20 * np.log10(T)) + 1) / 20.0)).astype(np.int64))
    return t[(t >= 1) & (t <= T)]


def sweep(L: int = 8192, r_values=None, T: int = 100000, chunk: int = 500, seed: int = 1,
          layout: str = "bitpack", K: float = 0.5) -> dict:
    import torch
    from . import build, pgg
    build.build()
    if r_values is None:
        r_values = np.round(np.arange(3.730, 3.7601, 0.002), 6)
    r_values = np.asarray(r_values, dtype=np.float64)
    n = len(r_values)
    times = log_times(T)
    streams = [torch.cuda.Stream() for _ in range(n)]
    lats = []
    for i, r in enumerate(r_values):
        lat = pgg.Lattice(L, float(r), K, layout=layout, stream=streams[i].cuda_stream)
        lat.seed(seed + i, 0.5)
        lats.append(lat)
    if L >= 1024:
        lats[0].autotune(2)  # process-wide choice for (device, L, layout); restores the state
    counts = torch.zeros((n, chunk), dtype=torch.int64, device="cuda")
    rho = np.full((n, len(times)), np.nan)
    N = float(L) * L
    done = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    t0 = time.perf_counter()
    while done < T:
        m = min(chunk, T - done)
        for i in range(n):
            with torch.cuda.stream(streams[i]):
                lats[i].step_mcs(m, counts[i].data_ptr())
        torch.cuda.synchronize()
        c = counts[:, :m].cpu().numpy()
        sel = (times > done) & (times <= done + m)
        if sel.any():
            rho[:, sel] = c[:, times[sel] - done - 1] / N
        done += m
    ev1.record()
    torch.cuda.synchronize()
    gpu_s = ev0.elapsed_time(ev1) / 1e3
    wall = time.perf_counter() - t0
    for lat in lats:
        lat.close()
    return {"L": L, "K": K, "T": T, "r": r_values.tolist(), "t": times.tolist(), "rho": rho.tolist(),
            "gpu_s": gpu_s, "wall_s": wall,
            "site_updates_per_s": n * N * T / gpu_s, "schedule": None}


def analyse(res: dict, t_min_frac: float = 0.01, late_frac: float = 0.3,
            rho_floor: float = 2e-3) -> dict:
    """Late-time log-log slope of rho_C(t) for every r, and a fit of the late-time density to
    rho = A (r - r_c)^beta (Eq. (5)) over the r whose density stays above rho_floor."""
    t = np.asarray(res["t"], dtype=np.float64)
    rho = np.asarray(res["rho"], dtype=np.float64)
    r = np.asarray(res["r"], dtype=np.float64)
    T = t.max()
    sel = t >= t_min_frac * T
    per_r = []
    late = np.full(len(r), np.nan)
    for i in range(len(r)):
        y, x = rho[i, sel], t[sel]
        ok = y > 0
        slope = float(np.polyfit(np.log(x[ok]), np.log(y[ok]), 1)[0]) if ok.sum() >= 3 else None
        lw = t >= late_frac * T
        late[i] = float(np.nanmean(rho[i, lw]))
        per_r.append({"r": float(r[i]), "late_slope": slope, "rho_late": late[i],
                      "rho_T": float(rho[i, -1])})
    use = late > rho_floor
    fit = fit_power_law(r[use], late[use], window=0.03)
    return {"per_r": per_r, "power_law_fit": fit,
            "paper": {"r_c": 3.7443, "beta": 0.56, "beta_dp": 0.584}}


def fit_power_law(r, rho, window: float = 0.02, r_c_fixed: float = 3.7443):
    """Least-squares fit of log rho = beta log(r - r_c) + log A (Eq. (5)) over points with
    rho > 0: r_c scanned in steps of 1e-5 over the `window` below the smallest r; also beta
    with r_c fixed at the paper's value. None with fewer than 3 points."""
    r = np.asarray(r, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > 0
    if ok.sum() < 3:
        return None
    rs, ys = r[ok], np.log(rho[ok])
    best = None
    for rc in np.arange(rs.min() - window, rs.min() - 1e-5, 1e-5):
        X = np.log(rs - rc)
        beta, logA = np.polyfit(X, ys, 1)
        resid = float(np.sum((ys - (beta * X + logA)) ** 2))
        if best is None or resid < best[0]:
            best = (resid, rc, beta, logA)
    fixed = float(np.polyfit(np.log(rs - r_c_fixed), ys, 1)[0]) if rs.min() > r_c_fixed else None
    return {"r_c": float(best[1]), "beta": float(best[2]), "A": float(np.exp(best[3])), "residual": best[0],
            "points": int(ok.sum()), "beta_with_paper_r_c": fixed}


def anneal_scan(L: int = 2048, r_values=None, T_relax: int = 100000, T_meas: int = 100000,
                seed: int = 1, K: float = 0.5, chunk: int = 5000, layout: str = "bitpack") -> dict:
    """Stationary cooperator density by annealing (Section V's procedure for the stationary
    state): one lattice, started from Bernoulli(1/2) at the largest r, is carried down the r
    values in decreasing order; at each r it relaxes for T_relax MCS (discarded) and is then
    averaged over T_meas MCS. Starting each r from the state of the previous one avoids the
    collapse-and-recovery transient of a random start."""
    import torch
    from . import build, pgg
    build.build()
    if r_values is None:
        r_values = np.round(np.arange(3.800, 3.7479, -0.004), 6)
    r_values = np.sort(np.asarray(r_values, dtype=np.float64))[::-1]
    stream = torch.cuda.current_stream()
    counts = torch.zeros(chunk, dtype=torch.int64, device="cuda")
    N = float(L) * L
    out = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with pgg.Lattice(L, float(r_values[0]), K, layout=layout, stream=stream.cuda_stream) as lat:
        lat.seed(seed, 0.5)
        if L >= 1024:
            lat.autotune(2)
        torch.cuda.synchronize()
        ev0.record(stream)
        for r in r_values:
            lat.set_params(float(r), K)
            lat.advance(T_relax)
            total, sq, done, last = 0.0, 0.0, 0, 0
            while done < T_meas:
                m = min(chunk, T_meas - done)
                lat.step_mcs(m, counts.data_ptr())
                c = counts[:m].double() / N
                total += float(c.sum())
                sq += float((c * c).sum())
                last = float(c[-1])
                done += m
            mean = total / T_meas
            out.append({"r": float(r), "rho": mean, "rho_std": float(np.sqrt(max(sq / T_meas - mean * mean, 0.0))),
                        "rho_end": last, "absorbed": last == 0.0})
        ev1.record(stream)
        torch.cuda.synchronize()
    res = {"L": L, "K": K, "T_relax": T_relax, "T_meas": T_meas, "seed": seed, "points": out,
           "gpu_s": ev0.elapsed_time(ev1) / 1e3}
    # fit rho = A (r - r_c)^beta over the surviving points, with r_c free and with the paper's r_c
    res["fit"] = fit_power_law([p["r"] for p in out], [p["rho"] for p in out])
    res["paper"] = {"r_c": 3.7443, "beta": 0.56}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=8192)
    ap.add_argument("--T", type=int, default=100000)
    ap.add_argument("--layout", default="bitpack")
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--r-lo", type=float, default=3.730)
    ap.add_argument("--r-hi", type=float, default=3.760)
    ap.add_argument("--r-step", type=float, default=0.002)
    ap.add_argument("--anneal", action="store_true",
                    help="stationary densities by annealing down in r (T relaxation + T averaging per r)")
    args = ap.parse_args()
    r_values = np.round(np.arange(args.r_lo, args.r_hi + 0.5 * args.r_step, args.r_step), 6)
    if args.anneal:
        print(json.dumps(anneal_scan(args.L, r_values, T_relax=args.T, T_meas=args.T, layout=args.layout)))
        return
    res = sweep(args.L, r_values=r_values, T=args.T, layout=args.layout, chunk=args.chunk)
    res["analysis"] = analyse(res)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
