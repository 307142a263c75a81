"""The late-time power-law fit of the critical sweep recovers a known (r_c, beta)."""
import numpy as np

from paper_1704_08098_gb300 import critical


def test_power_law_fit_recovers_known_exponent():
    r = np.round(np.arange(3.730, 3.7601, 0.002), 6)
    t = critical.log_times(100000)
    rc, beta, A = 3.7443, 0.56, 1.9
    rho = np.zeros((len(r), len(t)))
    for i, ri in enumerate(r):
        if ri > rc:
            rho[i] = A * (ri - rc) ** beta          # stationary from the start
        else:
            rho[i] = 0.5 * t.astype(float) ** -1.5   # decaying
    res = {"r": r.tolist(), "t": t.tolist(), "rho": rho.tolist()}
    fit = critical.analyse(res, rho_floor=1e-3)["power_law_fit"]
    assert abs(fit["r_c"] - rc) < 2e-4
    assert abs(fit["beta"] - beta) < 0.02


def test_log_times_are_log_spaced_and_unique():
    t = critical.log_times(100000)
    assert t[0] == 1 and t[-1] == 100000
    assert np.all(np.diff(t) > 0)
    assert len(t) <= 101


def test_direct_fit_recovers_known_exponent_and_fixed_rc_slope():
    r = np.round(np.arange(3.748, 3.8001, 0.004), 6)
    rho = 1.3 * (r - 3.7443) ** 0.58
    fit = critical.fit_power_law(r, rho)
    assert abs(fit["r_c"] - 3.7443) < 2e-4 and abs(fit["beta"] - 0.58) < 0.01
    assert abs(fit["beta_with_paper_r_c"] - 0.58) < 1e-9
    assert critical.fit_power_law(r[:2], rho[:2]) is None
