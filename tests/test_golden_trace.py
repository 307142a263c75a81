"""The oracle's trajectory for the L = 64, r = 4, K = 0.5, seed 1 workload against the stored
counts of tests/golden/rho_trace_L64_counts.txt (written by make_rho_trace_L64.py from the oracle):
a regression fixture, so that a change moving the oracle, and with it the GPU parity target, is seen.
The GPU side is compared with the same file in tests/test_gpu_parity.py."""
import os

import numpy as np

import oracle
from paper_1704_08098_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rho_trace_L64_counts.txt")


def load_trace(path=GOLDEN):
    with open(path) as f:
        rows = [line for line in f if not line.startswith("#") and line.strip()]
    return np.array([int(x) for x in rows], dtype=np.uint64)


def test_oracle_reproduces_the_stored_trace():
    w = inputs.WORKLOADS["rho_trace_L64"]
    want = load_trace()
    assert len(want) == w["n_mcs"]
    o = oracle.Oracle()
    lat = o.init(w["L"], w["seed"], w["p"])
    got = o.run(lat, w["r"], w["K"], w["seed"], 0, w["n_mcs"])
    assert np.array_equal(got, want)
    # the run is neither absorbed nor frozen: the counts move and stay inside (0, L^2)
    assert 0 < int(want.min()) and int(want.max()) < w["L"] ** 2 and len(set(want.tolist())) > 100


def test_pairwise_oracle_reproduces_the_stored_trace():
    path = os.path.join(os.path.dirname(GOLDEN), "pair_trace_L64_counts.txt")
    want = load_trace(path)
    assert len(want) == 600
    o = oracle.Oracle()
    lat = o.init(64, 1, 0.5)
    got = o.pair_run(lat, (1.0, 0.0, 1.04, 0.0), 0.1, 1, 0, 600)
    assert np.array_equal(got, want)
    assert 0 < int(want.min()) and int(want.max()) < 64 ** 2 and len(set(want.tolist())) > 50
