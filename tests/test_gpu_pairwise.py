"""GPU parity for the pairwise game (Section VI): every kernel family, through the C ABI,
against the CPU oracle's pairwise dynamics, bit for bit.

The pairwise game runs on the same schedule and random stream as the group game; only
the payoff (a 2x2 matrix game with each nearest neighbour) and so the read radius (2 instead
of 3) differ. Lattices, counts and thresholds are exact, so every comparison is equality.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1704_08098_gb300 import inputs

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))

WEAK_PD = (1.0, 0.0, 1.04, 0.0)       # weak prisoner's dilemma, b = 1.04
SNOWDRIFT = (1.0, 0.5, 1.5, 0.0)
GENERIC = (3.0, -1.0, 5.0, 0.5)
MATRICES = {"weak_pd": (WEAK_PD, 0.1), "snowdrift": (SNOWDRIFT, 0.5), "generic": (GENERIC, 2.0)}


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


@pytest.fixture(scope="module")
def pgg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1704_08098_gb300 import build, pgg as P
    build.build()
    return P


def run_gpu(P, L, pay, K, seed, n_mcs, layout, schedule=None, lattice=None, step=0, p=0.5):
    with P.Lattice(L, 4.0, K, layout=layout) as lat:
        lat.set_game("pairwise", pay)
        if schedule:
            lat.set_schedule(**schedule)
        lat.seed(seed, p)
        if lattice is not None:
            lat.set(lattice, step)
        counts = lat.step_mcs(n_mcs)
        final, k = lat.get()
    return final, counts, k


def run_oracle(o, L, pay, K, seed, n_mcs, lattice=None, step=0, p=0.5):
    lat = o.init(L, seed, p) if lattice is None else np.ascontiguousarray(lattice, np.uint8).copy()
    counts = o.pair_run(lat, pay, K, seed, step, n_mcs, threads=THREADS)
    return lat, counts


def test_pair_threshold_table_matches_oracle(o, pgg):
    for pay, K in list(MATRICES.values()) + [((1.0, 0.0, 1.5, 0.0), 1e-6), ((0.7, -0.3, 1.9, 0.1), 1e6),
                                              ((2.0, 2.0, 2.0, 2.0), 0.4)]:
        with pgg.Lattice(64, 4.0, K) as lat:
            lat.set_game("pairwise", pay)
            assert lat.game() == ("pairwise", tuple(pay))
            T = lat.threshold_table().reshape(-1)
        assert not T[50:].any()
        for sx in (0, 1):
            sy = 1 - sx
            for nx in range(5):
                for ny in range(5):
                    want = o.threshold(o.pair_payoff_total(sx, nx, pay), o.pair_payoff_total(sy, ny, pay), K)
                    assert int(T[(sx * 5 + nx) * 5 + ny]) == want, (pay, K, sx, nx, ny)


SCHEDULES = {
    "simple": dict(kernel="simple"),
    "tiled_k1": dict(kernel="tiled", steps_per_launch=1),
    "tiled_k2": dict(kernel="tiled", steps_per_launch=2, tile_x=64, tile_y=32),
    "tiled_k4": dict(kernel="tiled", steps_per_launch=4, tile_x=128, tile_y=64),
    "tiled_k8": dict(kernel="tiled", steps_per_launch=8),
    "tiled_k16": dict(kernel="tiled", steps_per_launch=16, tile_x=64, tile_y=64),
}


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("sched", sorted(SCHEDULES))
@pytest.mark.parametrize("game", sorted(MATRICES))
def test_pair_L64_all_schedules(o, pgg, layout, sched, game):
    pay, K = MATRICES[game]
    want_lat, want_counts = run_oracle(o, 64, pay, K, 11, 200)
    got_lat, got_counts, k = run_gpu(pgg, 64, pay, K, 11, 200, layout, SCHEDULES[sched])
    assert k == 16 * 200
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("L,tx,ty,k", [(192, 128, 36, 4), (320, 256, 100, 8), (128, 64, 124, 16),
                                        (256, 192, 60, 2)])
def test_pair_tiled_ragged_tiles(o, pgg, layout, L, tx, ty, k):
    """Tiles that do not divide L, with the pairwise game's 2k-site halo."""
    want_lat, want_counts = run_oracle(o, L, GENERIC, 2.0, 5 + L, 12)
    got_lat, got_counts, _ = run_gpu(pgg, L, GENERIC, 2.0, 5 + L, 12, layout,
                                     dict(kernel="tiled", steps_per_launch=k, tile_x=tx, tile_y=ty))
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("L", [36, 100, 4])
def test_pair_ragged_u8_simple(o, pgg, L):
    want_lat, want_counts = run_oracle(o, L, SNOWDRIFT, 0.5, 3, 25)
    got_lat, got_counts, _ = run_gpu(pgg, L, SNOWDRIFT, 0.5, 3, 25, "u8", dict(kernel="simple"))
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


DIRECT = {"direct4": dict(kernel="direct", tile_x=4, tile_y=128), "direct8": dict(kernel="direct", tile_x=8, tile_y=64)}


@pytest.mark.parametrize("sched", sorted(DIRECT))
@pytest.mark.parametrize("L", [256, 768])
def test_pair_direct_kernel(o, pgg, sched, L):
    want_lat, want_counts = run_oracle(o, L, WEAK_PD, 0.1, 70 + L, 12)
    got_lat, got_counts, _ = run_gpu(pgg, L, WEAK_PD, 0.1, 70 + L, 12, "bitpack", DIRECT[sched])
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L,n_mcs", [(256, 10), (1024, 6), (4096, 2)])
def test_pair_resident_kernel(o, pgg, L, n_mcs, layout):
    want_lat, want_counts = run_oracle(o, L, SNOWDRIFT, 0.5, 90 + L, n_mcs)
    got_lat, got_counts, k = run_gpu(pgg, L, SNOWDRIFT, 0.5, 90 + L, n_mcs, layout, dict(kernel="resident"))
    assert k == 16 * n_mcs
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L,spe,n_mcs", [(1024, 1, 5), (2048, 2, 3), (2048, 4, 3)])
def test_pair_resident_steps_per_exchange(o, pgg, L, spe, n_mcs, layout):
    """The pairwise game on the resident kernel with 1, 2 or 4 steps per halo exchange (halo of
    2 rows per step: the game reads one line less, Section VI)."""
    want_lat, want_counts = run_oracle(o, L, SNOWDRIFT, 0.5, 95 + L + spe, n_mcs)
    got_lat, got_counts, k = run_gpu(pgg, L, SNOWDRIFT, 0.5, 95 + L + spe, n_mcs, layout,
                                     dict(kernel="resident", tile_y=spe))
    assert k == 16 * n_mcs
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
def test_pair_full_size_default_schedule(o, pgg, layout):
    """L = 8192 (bit-packed) / 4096 (uint8) in the default (tuned) launch configuration."""
    L, n = (8192, 1) if layout == "bitpack" else (4096, 2)
    want_lat, want_counts = run_oracle(o, L, WEAK_PD, 0.1, 1, n)
    with pgg.Lattice(L, 4.0, 0.1, layout=layout) as lat:
        lat.set_game("pairwise", WEAK_PD)
        lat.seed(1)
        lat.autotune(1)
        got_counts = lat.step_mcs(n)
        got_lat, _ = lat.get()
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


def test_pair_long_run_L8192_one_mcs_per_call(o, pgg):
    """The pairwise benchmark's configuration (L = 8192 bit-packed, weak prisoner's dilemma,
    K = 0.1, the resident kernel, one call per MCS) for its first 40 MCS."""
    L, n = 8192, 40
    want_lat, want_counts = run_oracle(o, L, WEAK_PD, 0.1, 3, n)
    with pgg.Lattice(L, 4.0, 0.1, layout="bitpack") as lat:
        lat.set_game("pairwise", WEAK_PD)
        lat.set_schedule("resident")
        lat.seed(3)
        got_counts = np.concatenate([lat.step_mcs(1) for _ in range(n)])
        got_lat, _ = lat.get()
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


def test_pair_structured_inputs_and_game_switching(o, pgg):
    """A clustered start, switching game and kernel between calls: each call plays the game
    set at the time, on the state the previous call left."""
    L = 512
    lat0 = inputs.clustered_lattice(L, 30, 14, seed=4)
    ref = lat0.copy()
    k = 16 * 3
    want = [o.pair_run(ref, GENERIC, 2.0, 9, k, 3, threads=THREADS)]
    k += 16 * 3
    want.append(o.run(ref, 3.9, 2.0, 9, k, 2, threads=THREADS))
    k += 16 * 2
    want.append(o.pair_run(ref, GENERIC, 2.0, 9, k, 4, threads=THREADS))
    k += 16 * 4
    with pgg.Lattice(L, 3.9, 2.0, layout="bitpack") as lat:
        lat.seed(9)
        lat.set(lat0, 16 * 3)
        lat.set_game("pairwise", GENERIC)
        lat.set_schedule("direct", 1, 8)
        c1 = lat.step_mcs(3)
        lat.set_game("group")
        assert lat.game()[0] == "group"
        lat.set_schedule("tiled", 4, 128, 64)
        c2 = lat.step_mcs(2)
        lat.set_game("pairwise", GENERIC)
        lat.set_schedule("resident")
        c3 = lat.step_mcs(4)
        got, step = lat.get()
    assert step == k
    assert np.array_equal(np.concatenate([c1, c2, c3]), np.concatenate(want))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
def test_pair_absorbing_and_equal_payoffs(o, pgg, layout):
    for p in (0.0, 1.0):
        with pgg.Lattice(128, 4.0, 0.5, layout=layout) as lat:
            lat.set_game("pairwise", WEAK_PD)
            lat.seed(2, p)
            counts = lat.step_mcs(5)
        assert all(int(c) == int(p * 128 * 128) for c in counts)
    # R = S = T = P: every adoption is a fair coin flip
    want_lat, want_counts = run_oracle(o, 128, (2.0, 2.0, 2.0, 2.0), 0.3, 6, 20)
    got_lat, got_counts, _ = run_gpu(pgg, 128, (2.0, 2.0, 2.0, 2.0), 0.3, 6, 20, layout)
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


def test_set_game_rejects_bad_arguments(pgg):
    with pgg.Lattice(64, 4.0, 0.5) as lat:
        with pytest.raises(pgg.PGGError):
            lat.set_game("pairwise", None)
        with pytest.raises(pgg.PGGError):
            lat.set_game("pairwise", (1.0, float("nan"), 1.5, 0.0))
        assert lat.game()[0] == "group"
