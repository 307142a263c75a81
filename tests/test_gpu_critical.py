"""The concurrent critical-decay sweep records the same trajectories as separate runs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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
