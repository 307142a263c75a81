"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only produces lattices and
parameter sets from numpy's seeded generator, so that the CUDA library and the
CPU oracle can be driven with identical inputs. Initial conditions drawn by the
method itself (Section III: each site C or D with probability 1/2) are not made
here; both sides draw those from the Philox stream they each implement.
"""
from __future__ import annotations

import numpy as np


def random_lattice(L: int, p: float, seed: int) -> np.ndarray:
    """L x L uint8 lattice, each site 1 (cooperator) with probability p."""
    rng = np.random.default_rng(seed)
    return (rng.random((L, L)) < p).astype(np.uint8)


def clustered_lattice(L: int, n_blobs: int, radius: int, seed: int) -> np.ndarray:
    """L x L lattice of cooperator discs on a defector background (periodic),
    the compact-cluster structure the game forms (Section V)."""
    rng = np.random.default_rng(seed)
    lat = np.zeros((L, L), dtype=np.uint8)
    ii, jj = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    for _ in range(n_blobs):
        ci, cj = rng.integers(0, L, size=2)
        di = np.minimum(np.abs(ii - ci), L - np.abs(ii - ci))
        dj = np.minimum(np.abs(jj - cj), L - np.abs(jj - cj))
        lat[di * di + dj * dj <= radius * radius] = 1
    return lat


def uniform_params(n: int, r_lo: float, r_hi: float, seed: int) -> np.ndarray:
    """n synergy factors r drawn uniformly from [r_lo, r_hi]."""
    return np.random.default_rng(seed).uniform(r_lo, r_hi, size=n)


def replica_sizes(n: int, choices, seed: int) -> np.ndarray:
    """n lattice sizes drawn uniformly from ``choices``."""
    return np.random.default_rng(seed).choice(np.asarray(choices), size=n)


def mlp_init_params(seed: int, n_in: int = 202, n_hidden: int = 128, n_out: int = 2) -> np.ndarray:
    """Initial surrogate parameters (float32, packed W1, b1, W2, b2, W3, b3): weights uniform
    in +-sqrt(6 / fan_in) (He-uniform), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def random_features(B: int, seed: int, n_in: int = 202) -> np.ndarray:
    """B random surrogate inputs: 200 cooperator fractions in [0, 1] then normalised r, K."""
    rng = np.random.default_rng(seed)
    X = rng.random((B, n_in)).astype(np.float32)
    X[:, -2:] = rng.uniform(-1, 1, size=(B, 2)).astype(np.float32)
    return X


def random_labels(B: int, seed: int) -> np.ndarray:
    """B random (absorbed, stationary rho, mask) label rows."""
    rng = np.random.default_rng(seed)
    y = (rng.random(B) < 0.5).astype(np.float32)
    rho = np.where(y > 0, 0.0, rng.random(B)).astype(np.float32)
    return np.stack([y, rho, 1.0 - y], axis=1).astype(np.float32)


# Workloads used by the tests and the benchmark (sizes and parameters of
# the paper's experiments: Section V, Fig. 4 and Fig. 5).
WORKLOADS = {
    "rho_trace_L64": dict(L=64, r=4.0, K=0.5, p=0.5, seed=1, n_mcs=1000),
    "throughput_L4096": dict(L=4096, r_values=(3.5, 3.7, 3.9, 4.5, 5.0), K=0.5, p=0.5,
                             n_mcs=20000, window=5000),
    "critical_L8192": dict(L=8192, r=3.744, K=0.5, p=0.5, seed=1),
    "paper_timing_r398": dict(r=3.98, K=0.5, p=0.5),
}
