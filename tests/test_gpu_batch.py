"""GPU parity of the batched replica engine against the CPU oracle (bit for bit)."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_08098_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


@pytest.fixture(scope="module")
def pgg():
    import torch
    assert torch.cuda.is_available()
    from paper_1704_08098_gb300 import build, pgg as P
    build.build()
    return P


def mixed_batch(n, seed):
    L = inputs.replica_sizes(n, (64, 128, 256, 512, 1024), seed)
    r = inputs.uniform_params(n, 3.5, 4.2, seed + 1)
    return L, r, np.arange(100, 100 + n, dtype=np.uint64)


def oracle_replica(o, L, r, seed, n_mcs, step0=0, lattice=None):
    lat = o.init(L, seed, 0.5) if lattice is None else lattice.copy()
    counts = o.run(lat, r, 0.5, seed, step0, n_mcs, threads=THREADS)
    return lat, counts


def test_batch_matches_oracle(o, pgg):
    L, r, seeds = mixed_batch(14, 3)
    L[:5] = [64, 128, 256, 512, 1024]  # every size class present
    with pgg.Batch(L, r, 0.5, seeds) as b:
        b.seed(0.5)
        counts = b.step_mcs(4)
        for i in range(b.n):
            got, step = b.get(i)
            want, wc = oracle_replica(o, int(L[i]), float(r[i]), int(seeds[i]), 4)
            assert step == 64
            assert np.array_equal(counts[i], wc.astype(np.uint32)), i
            assert np.array_equal(got, want), i


@pytest.mark.parametrize("cta,warps", [(1024, [1, 1, 2, 8, 32]), (1024, [1, 2, 4, 16, 32]),
                                       (512, [1, 1, 2, 8, 16]), (512, [1, 1, 1, 4, 8])])
def test_batch_schedule_independent(pgg, cta, warps):
    L, r, seeds = mixed_batch(20, 8)
    ref = None
    with pgg.Batch(L, r, 0.5, seeds) as b:
        b.set_cta_threads(cta)
        b.set_team_warps(warps)
        b.seed(0.5)
        counts = b.step_mcs(5)
        lats = [b.get(i)[0] for i in range(b.n)]
    with pgg.Batch(L, r, 0.5, seeds) as b:
        b.seed(0.5)
        ref_counts = b.step_mcs(5)
        ref = [b.get(i)[0] for i in range(b.n)]
    assert np.array_equal(counts, ref_counts)
    assert all(np.array_equal(x, y) for x, y in zip(lats, ref))


def test_batch_graph_replay_continues(pgg):
    L, r, seeds = mixed_batch(10, 5)
    with pgg.Batch(L, r, 0.5, seeds) as g, pgg.Batch(L, r, 0.5, seeds) as d:
        d.use_graph(False)
        g.seed(0.5)
        d.seed(0.5)
        parts = [g.step_mcs(3) for _ in range(3)]   # one captured graph, replayed
        whole = d.step_mcs(9)
        assert np.array_equal(np.concatenate(parts, axis=1), whole)
        for i in range(g.n):
            a, ka = g.get(i)
            c, kc = d.get(i)
            assert ka == kc == 16 * 9 and np.array_equal(a, c)


def test_batch_matches_single_lattice_path(pgg):
    L, r, seeds = mixed_batch(6, 11)
    with pgg.Batch(L, r, 0.5, seeds) as b:
        b.seed(0.5)
        counts = b.step_mcs(7)
        for i in range(b.n):
            with pgg.Lattice(int(L[i]), float(r[i]), 0.5, layout="bitpack") as s:
                s.seed(int(seeds[i]), 0.5)
                c = s.step_mcs(7)
                lat, _ = s.get()
            assert np.array_equal(c.astype(np.uint32), counts[i])
            assert np.array_equal(lat, b.get(i)[0])


def test_batch_set_lattice_and_autotune(o, pgg):
    L = np.array([256, 64, 1024, 512], dtype=np.int32)
    r = np.array([3.7, 4.0, 3.9, 3.8])
    seeds = np.array([5, 6, 7, 8], dtype=np.uint64)
    with pgg.Batch(L, r, 0.5, seeds) as b:
        b.seed(0.5)
        lat0 = inputs.clustered_lattice(256, 6, 10, seed=2)
        b.set(0, lat0, 16 * 3)
        before = [b.get(i) for i in range(b.n)]
        best = b.autotune(2)
        assert len(best["team_warps"]) == 5 and best["ms"] > 0
        after = [b.get(i) for i in range(b.n)]
        for (x, kx), (y, ky) in zip(before, after):
            assert kx == ky and np.array_equal(x, y)
        counts = b.step_mcs(3)
        got, step = b.get(0)
    want, wc = oracle_replica(o, 256, 3.7, 5, 3, step0=16 * 3, lattice=lat0)
    assert step == 16 * 6 and np.array_equal(got, want)
    assert np.array_equal(counts[0], wc.astype(np.uint32))


def test_batch_rejects_unsupported_sizes(pgg):
    with pytest.raises(pgg.PGGError):
        pgg.Batch([64, 96], [4.0, 4.0], 0.5, [1, 2])
    with pytest.raises(pgg.PGGError):
        pgg.Batch([2048], [4.0], 0.5, [1])


@pytest.mark.parametrize("p,r", [(0.5, 1.5), (1.0, 4.0), (0.0, 4.0)], ids=["decays", "all-C", "all-D"])
def test_batch_absorbed_replicas(o, pgg, p, r):
    """A replica whose count reaches 0 or L^2 stops being updated: its later counts, its lattice
    and its step counter still equal the oracle's full run, in both halves of a call and across
    calls (r = 1.5 takes a random start to all-D within a few MCS; all-C and all-D starts are
    absorbing from the first MCS)."""
    L = np.array([64, 64, 128, 256], dtype=np.int32)
    seeds = np.arange(40, 44, dtype=np.uint64)
    n_mcs = 40
    with pgg.Batch(L, np.full(4, r), 0.5, seeds) as b:
        b.seed(p)
        first = b.step_mcs(n_mcs)
        second = b.step_mcs(n_mcs)
        for i in range(4):
            got, step = b.get(i)
            lat = o.init(int(L[i]), int(seeds[i]), p)
            want = o.run(lat, r, 0.5, int(seeds[i]), 0, 2 * n_mcs, threads=THREADS)
            assert step == 32 * n_mcs
            assert np.array_equal(np.concatenate([first[i], second[i]]), want.astype(np.uint32)), i
            assert np.array_equal(got, lat), i
            if p != 0.5:
                assert want[0] in (0, int(L[i]) ** 2)
    if p == 0.5:
        assert want[n_mcs - 1] == 0  # the decaying replicas are absorbed within the first call
