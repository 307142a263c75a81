"""What the trained surrogate gains: an r_c bisection that stops replicas after 200 MCS when
the network is confident, against the plain bisection that simulates every probe to the end.
The full simulation judges every decision the network takes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    assert torch.cuda.is_available()
    from paper_1704_08098_gb300 import surrogate as S
    X, Y, meta = S.generate(n=3000, L=64, T_label=1500, window=300, chunk=300, seed=3,
                            r_lo=3.0, r_hi=5.0)
    assert 0.05 < meta["absorbed_frac"] < 0.95
    params, hist = S.train(X[:2700], Y[:2700], epochs=30, batch=256, lr=2e-3, seed=4)
    assert hist[-1] < hist[0]
    return params, S.evaluate(params, X[2700:], Y[2700:])


def test_surrogate_is_accurate_on_held_out_runs(trained):
    _, ev = trained
    assert ev["accuracy"] > 0.85
    assert ev["confident_frac"] > 0.3 and ev["confident_accuracy"] > 0.95


def test_surrogate_bisection_gains_and_is_judged_by_simulation(trained):
    from paper_1704_08098_gb300 import rc_search as R
    from paper_1704_08098_gb300.surrogate import Surrogate
    params, _ = trained
    kw = dict(L=128, lo=3.0, hi=5.0, width=0.06, T_max=3000, replicas=4, seed=77)
    plain = R.bisect(**kw)
    s = Surrogate(params)
    gated = R.bisect(surrogate=s, conf=0.95, **kw)
    s.close()
    decided = [p for p in gated["probes"] if p["decided_by"] == "surrogate"]
    assert decided, "the surrogate decided no probe"
    # the full simulation (same seeds) is the judge of every surrogate decision
    for k, p in enumerate(gated["probes"]):
        if p["decided_by"] == "surrogate":
            full = R.probe(p["r"], 128, 3000, 4, 77 + 1000 * k)
            assert full["absorbing"] == p["absorbing"], p
    assert gated["gpu_ms"] < plain["gpu_ms"]
    assert sum(p["mcs"] for p in gated["probes"]) < sum(p["mcs"] for p in plain["probes"])
    # both brackets are consistent with the simulation's own answer
    lo, hi = plain["bracket"]
    glo, ghi = gated["bracket"]
    assert max(lo, glo) <= min(hi, ghi) + 1e-12
