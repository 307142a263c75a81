"""The concurrent critical-decay sweep (Section V: one lattice per r, all advancing at once on
their own streams, rho_C recorded at log-spaced times) records exactly the oracle's
trajectories, and the same ones as separate single-lattice runs."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


def test_sweep_matches_oracle():
    """Every recorded count of every r equals the CPU oracle's count after that MCS (same seed
    seed + i, same Bernoulli(1/2) start, same steps). L = 1024 takes the sweep's autotuned
    schedule, and chunks of 50 MCS that do not divide T = 120 exercise the chunked readback."""
    import torch
    assert torch.cuda.is_available()
    from paper_1704_08098_gb300 import critical
    L, T, seed = 1024, 120, 5
    r_values = [3.70, 3.744, 3.78, 3.90]
    res = critical.sweep(L=L, r_values=r_values, T=T, chunk=50, seed=seed)
    t = np.asarray(res["t"])
    assert t[0] == 1 and t[-1] <= T and np.all(np.diff(t) > 0)
    got = np.rint(np.asarray(res["rho"]) * float(L) * L).astype(np.int64)
    o = oracle.Oracle()
    for i, r in enumerate(r_values):
        lat = o.init(L, seed + i, 0.5)
        want = o.run(lat, r, 0.5, seed + i, 0, T, threads=THREADS).astype(np.int64)
        assert np.array_equal(got[i], want[t - 1]), f"r = {r}: sweep counts differ from the oracle"


def test_sweep_matches_independent_runs():
    import torch
    assert torch.cuda.is_available()
    from paper_1704_08098_gb300 import critical, pgg
    r_values = [3.70, 3.74, 3.78, 3.82]
    res = critical.sweep(L=512, r_values=r_values, T=300, chunk=70, seed=9)
    t = np.asarray(res["t"])
    assert t[0] == 1 and t[-1] <= 300 and np.all(np.diff(t) > 0)
    rho = np.asarray(res["rho"])
    assert np.all((rho >= 0) & (rho <= 1))
    for i, r in enumerate(r_values):
        with pgg.Lattice(512, r, 0.5, layout="bitpack") as lat:
            lat.seed(9 + i, 0.5)
            c = lat.step_mcs(300)
        assert np.allclose(rho[i], c[t - 1] / 512.0 ** 2, rtol=0, atol=0)
    an = critical.analyse(res, t_min_frac=0.1)
    assert len(an["per_r"]) == 4 and "power_law_fit" in an
