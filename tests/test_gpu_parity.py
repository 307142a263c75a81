"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle, bit for bit.

Lattices, per-MCS cooperator counts and the threshold table are integer or exact
results, so every comparison is exact equality (the threshold table is built by
each side in IEEE double precision with the same libm, see the threshold rule in
include/pgg.h).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1704_08098_gb300 import inputs
from test_golden_trace import load_trace

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


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


def run_gpu(P, L, r, K, seed, n_mcs, layout, schedule=None, p=0.5, lattice=None, step=0):
    with P.Lattice(L, r, K, layout=layout) as lat:
        if schedule:
            lat.set_schedule(**schedule)
        if lattice is None:
            lat.seed(seed, p)
        else:
            lat.seed(seed, p)
            lat.set(lattice, step)
        counts = lat.step_mcs(n_mcs) if n_mcs else np.zeros(0, np.uint64)
        final, k = lat.get()
    return final, counts, k


def run_oracle(o, L, r, K, seed, n_mcs, p=0.5, lattice=None, step=0):
    lat = o.init(L, seed, p) if lattice is None else np.ascontiguousarray(lattice, np.uint8).copy()
    counts = o.run(lat, r, K, seed, step, n_mcs, threads=THREADS)
    return lat, counts


SCHEDULES = {
    "simple": dict(kernel="simple"),
    "tiled_k1": dict(kernel="tiled", steps_per_launch=1),
    "tiled_k2": dict(kernel="tiled", steps_per_launch=2, tile_x=64, tile_y=32),
    "tiled_k4": dict(kernel="tiled", steps_per_launch=4, tile_x=128, tile_y=64),
    "tiled_k8": dict(kernel="tiled", steps_per_launch=8),
    "tiled_k16": dict(kernel="tiled", steps_per_launch=16, tile_x=64, tile_y=64),
}


def test_threshold_table_matches_oracle(o, pgg):
    for r, K in ((4.0, 0.5), (3.7443, 0.5), (3.98, 0.5), (5.0, 0.1), (4.2, 1e-6), (3.5, 1e6),
                 (2.0, 3.3)):
        with pgg.Lattice(64, r, K) as lat:
            T = lat.threshold_table()
        for sx in (0, 1):
            sy = 1 - sx
            for Sx in range(26):
                for Sy in range(26):
                    want = o.threshold(o.payoff_total(sx, Sx, r), o.payoff_total(sy, Sy, r), K)
                    assert int(T[sx, Sx, Sy]) == want, (r, K, sx, Sx, Sy)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("L,p,seed", [(64, 0.5, 1), (96, 0.3, 7), (256, 0.5, 123), (32, 1.0, 2),
                                      (64, 0.0, 3)])
def test_initial_condition(o, pgg, layout, L, p, seed):
    with pgg.Lattice(L, 4.0, 0.5, layout=layout) as lat:
        lat.seed(seed, p)
        got, step = lat.get()
        count = lat.count()
    want = o.init(L, seed, p)
    assert step == 0
    assert np.array_equal(got, want)
    assert count == int(want.sum())


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("sched", sorted(SCHEDULES))
def test_rho_trace_L64_1000_mcs(o, pgg, layout, sched):
    """The L = 64, r = 4, K = 0.5, seed 1 workload: rho_C(t) per MCS for 1000 MCS."""
    w = inputs.WORKLOADS["rho_trace_L64"]
    want_lat, want_counts = run_oracle(o, w["L"], w["r"], w["K"], w["seed"], w["n_mcs"])
    got_lat, got_counts, k = run_gpu(pgg, w["L"], w["r"], w["K"], w["seed"], w["n_mcs"], layout,
                                     SCHEDULES[sched])
    assert k == 16 * w["n_mcs"]
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)
    assert np.array_equal(got_counts, load_trace())   # the stored oracle trace


@pytest.mark.parametrize("L", [4, 8, 12, 20, 36, 100])
def test_ragged_u8_sizes_simple(o, pgg, L):
    want_lat, want_counts = run_oracle(o, L, 3.9, 0.5, 11, 40)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.9, 0.5, 11, 40, "u8", dict(kernel="simple"))
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("L", [32, 96, 160])
def test_ragged_bitpack_sizes_simple(o, pgg, L):
    want_lat, want_counts = run_oracle(o, L, 4.1, 0.5, 12, 30)
    got_lat, got_counts, _ = run_gpu(pgg, L, 4.1, 0.5, 12, 30, "bitpack", dict(kernel="simple"))
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


TILED_RAGGED = [
    # L, tile_x, tile_y, k: tiles that do not divide L, single-tile lattices, deep fusion
    (192, 128, 40, 1), (192, 128, 40, 2), (320, 256, 96, 4), (448, 192, 68, 8),
    (128, 128, 128, 16), (64, 64, 4, 1), (64, 64, 8, 2), (576, 512, 100, 1),
]


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("L,tx,ty,k", TILED_RAGGED)
def test_tiled_ragged_tiles(o, pgg, layout, L, tx, ty, k):
    want_lat, want_counts = run_oracle(o, L, 3.8, 0.5, 5 + k, 12)
    sched = dict(kernel="tiled", steps_per_launch=k, tile_x=tx, tile_y=ty)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.8, 0.5, 5 + k, 12, layout, sched)
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
def test_structured_inputs(o, pgg, layout):
    """Clustered and sparse lattices set through the ABI, with a nonzero start step."""
    for lat0, step in ((inputs.clustered_lattice(128, 12, 9, seed=4), 16 * 77),
                       (inputs.random_lattice(128, 0.05, seed=5), 3),
                       (inputs.random_lattice(128, 0.95, seed=6), 16 * 1000 + 5)):
        want_lat, want_counts = run_oracle(o, 128, 3.74, 0.5, 99, 25, lattice=lat0, step=step)
        for sched in (dict(kernel="simple"), dict(kernel="tiled", steps_per_launch=4,
                                                  tile_x=64, tile_y=32)):
            got_lat, got_counts, k = run_gpu(pgg, 128, 3.74, 0.5, 99, 25, layout, sched,
                                             lattice=lat0, step=step)
            assert k == step + 16 * 25
            assert np.array_equal(got_counts, want_counts)
            assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("K", [1e-6, 0.5, 1e6])
def test_noise_limits(o, pgg, layout, K):
    want_lat, want_counts = run_oracle(o, 128, 4.0, K, 21, 20)
    got_lat, got_counts, _ = run_gpu(pgg, 128, 4.0, K, 21, 20, layout)
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
@pytest.mark.parametrize("p", [0.0, 1.0])
def test_absorbing_states_stay(pgg, layout, p):
    for sched in SCHEDULES.values():
        final, counts, _ = run_gpu(pgg, 128, 3.9, 0.5, 8, 10, layout, sched, p=p)
        assert final.sum() == (128 * 128 if p == 1.0 else 0)
        assert all(int(c) == int(final.sum()) for c in counts)


def test_zero_mcs_is_noop(pgg):
    with pgg.Lattice(64, 4.0, 0.5) as lat:
        lat.seed(3)
        before, k0 = lat.get()
        lat.step_mcs(0)
        after, k1 = lat.get()
    assert k0 == k1 == 0 and np.array_equal(before, after)


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
def test_checkpoint_resume_is_exact(pgg, layout):
    with pgg.Lattice(256, 3.9, 0.5, layout=layout) as a:
        a.seed(77)
        ca = a.step_mcs(40)
        full, ka = a.get()
    with pgg.Lattice(256, 3.9, 0.5, layout=layout) as b:
        b.seed(77)
        c1 = b.step_mcs(20)
        mid, kmid = b.get()
    with pgg.Lattice(256, 3.9, 0.5, layout=layout) as c:
        c.seed(77)
        c.set(mid, kmid)
        c2 = c.step_mcs(20)
        end, kc = c.get()
    assert ka == kc and np.array_equal(full, end)
    assert np.array_equal(ca, np.concatenate([c1, c2]))


@pytest.mark.parametrize("layout", ["u8", "bitpack"])
def test_packed_host_transfers(o, pgg, layout):
    """pgg_get/set_lattice_packed carry the same state as the uint8 transfers (bit b of word
    w = column 32w + b), and a run resumed from a packed checkpoint matches the oracle."""
    L = 256
    lat0 = inputs.random_lattice(L, 0.4, seed=21)
    words = (lat0.reshape(L, L // 32, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(-1)
    words = words.astype(np.uint32)
    with pgg.Lattice(L, 3.9, 0.5, layout=layout) as lat:
        lat.seed(5)
        lat.set_packed(words, 16 * 7)
        got, step = lat.get()
        assert step == 16 * 7 and np.array_equal(got, lat0)
        back, _ = lat.get_packed()
        assert np.array_equal(back, words)
        counts = lat.step_mcs(9)
        final, _ = lat.get()
        packed_final, _ = lat.get_packed()
    ref = lat0.copy()
    want = o.run(ref, 3.9, 0.5, 5, 16 * 7, 9, threads=THREADS)
    assert np.array_equal(counts, want) and np.array_equal(final, ref)
    bits = ((packed_final[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(L, L)
    assert np.array_equal(bits.astype(np.uint8), ref)


def pack_rows(lat):
    L = lat.shape[0]
    words = (lat.reshape(L, L // 32, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(-1)
    return words.astype(np.uint32)


@pytest.mark.parametrize("kernel", ["resident", "tiled", "direct"])
@pytest.mark.parametrize("layout", ["bitpack", "u8"])
def test_staged_uploads_overlap_steps(o, pgg, layout, kernel):
    """pgg_stage_lattice_packed in a loop (stage input i, step it with counts into device memory,
    read the counts back through pinned memory while the next input is staged): every input's
    trajectory matches the oracle run from that input and step."""
    import torch
    if kernel == "direct" and layout == "u8":
        pytest.skip("the direct kernel runs bit-packed lattices only")
    L, n_mcs = 512, 3
    lats = [inputs.random_lattice(L, p, seed=40 + i) for i, p in enumerate((0.5, 0.3, 0.7, 0.5, 0.45))]
    steps = [0, 16 * 5, 16 * 11 + 0, 7 * 16, 16 * 1000]
    host = [torch.from_numpy(pack_rows(x).reshape(-1).view(np.int32)).pin_memory() for x in lats]
    dev = torch.zeros((len(lats), n_mcs), dtype=torch.int64, device="cuda")
    back = torch.zeros((len(lats), n_mcs), dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream()
    with pgg.Lattice(L, 3.9, 0.5, layout=layout, stream=stream.cuda_stream) as lat:
        lat.set_schedule(kernel, 4 if kernel == "tiled" else 1)
        lat.seed(9)
        done = []
        for i in range(len(lats)):
            lat.stage_packed_from_pointer(host[i].data_ptr(), steps[i])
            assert lat.state()[1] == steps[i]
            lat.step_mcs(n_mcs, dev[i].data_ptr())
            back[i].copy_(dev[i], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
            done.append(ev)
        done[-1].synchronize()
        final, step = lat.get()
    assert step == steps[-1] + 16 * n_mcs
    for i, x in enumerate(lats):
        ref = x.copy()
        want = o.run(ref, 3.9, 0.5, 9, steps[i], n_mcs, threads=THREADS)
        assert np.array_equal(back[i].numpy().astype(np.uint64), want), i
    assert np.array_equal(final, ref)


def test_staged_lattice_is_applied_by_every_reader(o, pgg):
    """A staged lattice replaces the state at the next call that reads or writes it: get, count,
    a second stage before it is applied is refused, pgg_seed overwrites it, and a context
    destroyed with a staged lattice pending releases cleanly."""
    import torch
    L = 256
    a = inputs.random_lattice(L, 0.35, seed=3)
    b = inputs.random_lattice(L, 0.6, seed=4)
    ha = torch.from_numpy(pack_rows(a).reshape(-1).view(np.int32)).pin_memory()
    hb = torch.from_numpy(pack_rows(b).reshape(-1).view(np.int32)).pin_memory()
    for layout in ("bitpack", "u8"):
        with pgg.Lattice(L, 3.9, 0.5, layout=layout) as lat:
            lat.seed(2)
            lat.stage_packed_from_pointer(ha.data_ptr(), 48)
            assert lat.state() == (2, 48)
            with pytest.raises(pgg.PGGError) as e:
                lat.stage_packed_from_pointer(hb.data_ptr(), 0)
            assert e.value.status == pgg.PGG_ERR_STATE
            got, step = lat.get()
            assert step == 48 and np.array_equal(got, a)
            lat.stage_packed_from_pointer(hb.data_ptr(), 16)
            assert lat.count() == int(b.sum())
            assert np.array_equal(lat.get()[0], b)
            lat.stage_packed_from_pointer(ha.data_ptr(), 32)
            lat.seed(2, 0.5)   # overwrites the staged lattice
            seeded, step = lat.get()
            assert step == 0 and np.array_equal(seeded, o.init(L, 2, 0.5))
            lat.stage_packed_from_pointer(hb.data_ptr(), 64)   # left pending at destroy


def test_layouts_and_schedules_agree_L1024(pgg):
    ref = None
    for layout in ("u8", "bitpack"):
        for sched in SCHEDULES.values():
            final, counts, _ = run_gpu(pgg, 1024, 3.8, 0.5, 31, 6, layout, sched)
            if ref is None:
                ref = (final, counts)
            assert np.array_equal(final, ref[0]) and np.array_equal(counts, ref[1])


def test_counts_into_device_memory(pgg):
    import torch
    with pgg.Lattice(128, 4.0, 0.5, layout="bitpack") as lat:
        lat.seed(5)
        dev = torch.zeros(30, dtype=torch.int64, device="cuda")
        lat.step_mcs(30, dev.data_ptr())
        torch.cuda.synchronize()
        d = dev.cpu().numpy().astype(np.uint64)
    with pgg.Lattice(128, 4.0, 0.5, layout="bitpack") as lat:
        lat.seed(5)
        h = lat.step_mcs(30)
    assert np.array_equal(d, h)


@pytest.mark.parametrize("L,n_mcs,layout", [(4096, 3, "u8"), (4096, 3, "bitpack"),
                                            (8192, 2, "bitpack"), (8192, 1, "u8")])
def test_full_size_against_oracle(o, pgg, L, n_mcs, layout):
    """The paper's large lattices (Section V: up to 4096; 8192 here) in the default
    (tuned) launch configuration, the one the benchmark times."""
    want_lat, want_counts = run_oracle(o, L, 3.744, 0.5, 1, n_mcs)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.744, 0.5, 1, n_mcs, layout)
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("L,n_mcs", [(4096, 100), (8192, 50)])
def test_full_size_long_runs_one_mcs_per_call(o, pgg, L, n_mcs):
    """Long runs at the benchmark's sizes in its launch configuration (bit-packed, the resident
    kernel, one call and one launch per MCS): the count after every MCS and the final lattice
    equal the oracle's (the first 100 MCS at L = 4096 and 50 at L = 8192; the oracle is too slow
    for the full 2 x 10^4-MCS runs there)."""
    want_lat, want_counts = run_oracle(o, L, 3.744, 0.5, 7, n_mcs)
    with pgg.Lattice(L, 3.744, 0.5, layout="bitpack") as lat:
        lat.set_schedule("resident")
        lat.seed(7, 0.5)
        got_counts = np.concatenate([lat.step_mcs(1) for _ in range(n_mcs)])
        got_lat, step = lat.get()
    assert step == 16 * n_mcs
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


DIRECT = {"direct4": dict(kernel="direct", tile_x=4, tile_y=128), "direct8": dict(kernel="direct", tile_x=8, tile_y=64),
          "direct8b256": dict(kernel="direct", tile_x=8, tile_y=256)}


@pytest.mark.parametrize("sched", sorted(DIRECT))
@pytest.mark.parametrize("L", [256, 768, 1024])
def test_direct_kernel(o, pgg, sched, L):
    want_lat, want_counts = run_oracle(o, L, 3.9, 0.5, 40 + L, 15)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.9, 0.5, 40 + L, 15, "bitpack", DIRECT[sched])
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


def test_direct_kernel_structured_and_switching(o, pgg):
    """Set lattices mid-run and alternate kernels: the running cooperator count of the
    direct kernel must be re-established whenever another path changed the lattice."""
    L = 512
    lat0 = inputs.clustered_lattice(L, 30, 14, seed=9)
    ref = lat0.copy()
    want = []
    k = 16 * 5
    for n in (3, 2, 4):
        want.append(o.run(ref, 3.75, 0.5, 7, k, n, threads=THREADS))
        k += 16 * n
    with pgg.Lattice(L, 3.75, 0.5, layout="bitpack") as lat:
        lat.seed(7)
        lat.set(lat0, 16 * 5)
        lat.set_schedule("direct", 1, 4)
        c1 = lat.step_mcs(3)
        lat.set_schedule("tiled", 2, 128, 64)
        c2 = lat.step_mcs(2)
        lat.set_schedule("direct", 1, 8)
        c3 = lat.step_mcs(4)
        got, step = lat.get()
    assert step == k
    assert np.array_equal(np.concatenate([c1, c2, c3]), np.concatenate(want))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("layout,L", [("bitpack", 512), ("u8", 256), ("bitpack", 96)])
def test_autotune_restores_state_and_keeps_results(o, pgg, layout, L):
    """pgg_autotune times schedules on a saved copy and restores lattice, step and schedule;
    the tuned AUTO schedule gives the same trajectory as the oracle."""
    with pgg.Lattice(L, 3.85, 0.5, layout=layout) as lat:
        lat.seed(5)
        lat.step_mcs(2)
        before, k_before = lat.get()
        best = lat.autotune(1)
        after, k_after = lat.get()
        assert k_before == k_after and np.array_equal(before, after)
        assert best["kernel"] in ("resident", "direct", "tiled", "simple") and best["ms_per_mcs"] > 0
        counts = lat.step_mcs(6)
        final, _ = lat.get()
    ref = before.copy()
    want = o.run(ref, 3.85, 0.5, 5, k_before, 6, threads=THREADS)
    assert np.array_equal(counts, want) and np.array_equal(final, ref)


@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L,n_mcs", [(256, 12), (768, 6), (1024, 8), (4096, 2)])
def test_resident_kernel(o, pgg, L, n_mcs, layout):
    """Both layouts (a uint8 lattice runs on a packed copy for the call)."""
    want_lat, want_counts = run_oracle(o, L, 3.8, 0.5, 60 + L, n_mcs)
    got_lat, got_counts, k = run_gpu(pgg, L, 3.8, 0.5, 60 + L, n_mcs, layout, dict(kernel="resident"))
    assert k == 16 * n_mcs
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L,spe,n_mcs", [(1024, 1, 6), (1024, 2, 6), (2048, 4, 3), (2816, 2, 2), (4096, 4, 2),
                                         (4096, 1, 2)])
def test_resident_steps_per_exchange(o, pgg, L, spe, n_mcs, layout):
    """The resident kernel with its halo exchanged every 1, 2 or 4 sublattice steps (the halo
    rows updated redundantly in between) against the oracle; L = 2816 has bands of 18 and 19
    rows."""
    want_lat, want_counts = run_oracle(o, L, 3.8, 0.5, 70 + L + spe, n_mcs)
    got_lat, got_counts, k = run_gpu(pgg, L, 3.8, 0.5, 70 + L + spe, n_mcs, layout,
                                     dict(kernel="resident", tile_y=spe))
    assert k == 16 * n_mcs
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("spe", [1, 4])
def test_resident_dense_and_sparse_passes(o, pgg, spe):
    """A random half-and-half lattice (most sites can change: the dense pass) and a lattice of a
    few cooperator discs in a defector sea (few boundary sites: the pass over active sites only),
    each run for several MCS in one call and in calls of one MCS (the pass is chosen per step from
    the previous step's adoptions, across launches too), against the oracle."""
    L = 2048
    for lat0 in (inputs.random_lattice(L, 0.5, seed=71), inputs.clustered_lattice(L, 12, 20, seed=72)):
        ref = lat0.copy()
        want = o.run(ref, 3.8, 0.5, 13, 16 * 3, 4, threads=THREADS)
        with pgg.Lattice(L, 3.8, 0.5, layout="bitpack") as lat:
            lat.set_schedule("resident", 16, 0, spe)
            lat.seed(13)
            lat.set(lat0, 16 * 3)
            got = np.concatenate([lat.step_mcs(2), lat.step_mcs(1), lat.step_mcs(1)])
            final, _ = lat.get()
        assert np.array_equal(got, want) and np.array_equal(final, ref)


def test_resident_steps_per_exchange_limits(pgg):
    """Steps per exchange: 1, 2 or 4, and only as many as the bands' rows and the shared memory
    allow (bands of 6-7 rows at L = 1024 take at most 2); the default is the largest that fits."""
    with pgg.Lattice(1024, 3.8, 0.5, layout="bitpack") as lat:
        for bad in (3, 5, -1):
            with pytest.raises(pgg.PGGError):
                lat.set_schedule("resident", 16, 0, bad)
        with pytest.raises(pgg.PGGError):
            lat.set_schedule("resident", 16, 0, 4)
        lat.set_schedule("resident")
        assert lat.schedule()["tile_y"] == 2
    with pgg.Lattice(8192, 3.8, 0.5, layout="bitpack") as lat:
        lat.set_schedule("resident")
        assert lat.schedule()["tile_y"] == 4
        lat.set_schedule("resident", 16, 0, 1)
        assert lat.schedule()["tile_y"] == 1


def test_resident_full_size_and_resume(o, pgg):
    L = 8192
    want_lat, want_counts = run_oracle(o, L, 3.744, 0.5, 1, 2)
    with pgg.Lattice(L, 3.744, 0.5, layout="bitpack") as lat:
        lat.set_schedule("resident")
        lat.seed(1, 0.5)
        c1 = lat.step_mcs(1)
        c2 = lat.step_mcs(1)   # second launch continues from the stored state
        got, _ = lat.get()
    assert np.array_equal(np.concatenate([c1, c2]), want_counts)
    assert np.array_equal(got, want_lat)


def test_resident_largest_lattice_and_beyond(o, pgg):
    """The largest side whose bands still fit the shared memory (L = 14336: 94-95 rows of
    448 words per CTA) against the oracle; one side more that cannot be resident is refused
    (the direct kernel remains available for it)."""
    L = 14336
    want_lat, want_counts = run_oracle(o, L, 3.8, 0.5, 8, 1)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.8, 0.5, 8, 1, "bitpack", dict(kernel="resident"))
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)
    with pgg.Lattice(16384, 3.8, 0.5, layout="bitpack") as lat:
        with pytest.raises(pgg.PGGError):
            lat.set_schedule("resident")
        assert lat.schedule()["kernel"] == "direct"


@pytest.mark.parametrize("L", [16384, 32768])
def test_beyond_resident_sizes_default_schedule(o, pgg, L):
    """Lattices too large to be resident, up to the largest side the ABI accepts (32768:
    1.07e9 sites), in the default schedule (the direct kernel), one MCS against the oracle."""
    want_lat, want_counts = run_oracle(o, L, 3.9, 0.5, 3, 1)
    got_lat, got_counts, _ = run_gpu(pgg, L, 3.9, 0.5, 3, 1, "bitpack")
    assert np.array_equal(got_counts, want_counts)
    assert np.array_equal(got_lat, want_lat)


@pytest.mark.parametrize("kernel", ["resident", "direct", "tiled"])
def test_set_params_mid_run(o, pgg, kernel):
    """Changing r and K between calls (the annealing scan does) rebuilds the table for the next
    call only; the trajectory matches the oracle run in two legs."""
    L = 512
    ref = o.init(L, 23, 0.5)
    want = np.concatenate([o.run(ref, 4.2, 0.5, 23, 0, 4, threads=THREADS),
                           o.run(ref, 3.8, 0.3, 23, 16 * 4, 5, threads=THREADS)])
    with pgg.Lattice(L, 4.2, 0.5, layout="bitpack") as lat:
        lat.set_schedule(kernel, 4 if kernel == "tiled" else 1)
        lat.seed(23, 0.5)
        c1 = lat.step_mcs(4)
        lat.set_params(3.8, 0.3)
        c2 = lat.step_mcs(5)
        got, _ = lat.get()
    assert np.array_equal(np.concatenate([c1, c2]), want)
    assert np.array_equal(got, ref)


# step-kernel launches of one 3-MCS call: the resident kernel runs a whole call in one launch
@pytest.mark.parametrize("kernel,k,launches", [("resident", 16, 1), ("direct", 1, 48), ("tiled", 4, 12),
                                               ("simple", 1, 48)])
def test_kernel_timing_counts_step_launches(o, pgg, kernel, k, launches):
    """pgg_set_kernel_timing / pgg_kernel_time: one event pair per step-kernel launch, a positive
    duration no longer than the call took, and results unchanged."""
    import time
    L = 256
    ref = o.init(L, 4, 0.5)
    want = o.run(ref, 3.9, 0.5, 4, 0, 5, threads=THREADS)
    with pgg.Lattice(L, 3.9, 0.5, layout="bitpack") as lat:
        lat.set_schedule(kernel, k)
        lat.seed(4, 0.5)
        c1 = lat.step_mcs(2)
        lat.set_kernel_timing(True)
        t0 = time.perf_counter()
        c2 = lat.step_mcs(3)
        wall_ms = (time.perf_counter() - t0) * 1e3
        ms, n = lat.kernel_time()
        lat.set_kernel_timing(False)
        assert lat.kernel_time() == (0.0, 0)
        got, _ = lat.get()
    assert n == launches and 0.0 < ms <= wall_ms
    assert np.array_equal(np.concatenate([c1, c2]), want) and np.array_equal(got, ref)


def test_resident_many_launches(o, pgg):
    """2100 one-MCS calls on one context: the neighbour counters carry a per-launch base that
    wraps (and is reset) after 2047 launches; the trajectory must not notice."""
    L, n = 256, 2100
    want_lat, want_counts = run_oracle(o, L, 3.9, 0.5, 17, n)
    with pgg.Lattice(L, 3.9, 0.5, layout="bitpack") as lat:
        lat.set_schedule("resident")
        lat.seed(17, 0.5)
        counts = np.concatenate([lat.step_mcs(1) for _ in range(n)])
        got, step = lat.get()
    assert step == 16 * n
    assert np.array_equal(counts, want_counts)
    assert np.array_equal(got, want_lat)


def test_resident_wait_timeout_is_reported(o, pgg):
    """A bounded wait that runs out (spin limit 0: every wait gives up at once) returns
    PGG_ERR_TIMEOUT at the next synchronising call (the step call itself when it reads the counts
    back to the host); the context stays usable."""
    with pgg.Lattice(1024, 3.9, 0.5, layout="bitpack") as lat:
        lat.set_schedule("resident")
        lat.seed(3, 0.5)
        lat.set_spin_limit(0)
        lat.advance(1)
        with pytest.raises(pgg.PGGError) as exc:
            lat.count()
        assert exc.value.status == pgg.PGG_ERR_TIMEOUT
        lat.seed(3, 0.5)
        with pytest.raises(pgg.PGGError) as exc:   # with host counts, the step call reports it
            lat.step_mcs(1)
        assert exc.value.status == pgg.PGG_ERR_TIMEOUT
        lat.set_spin_limit(1 << 22)
        lat.seed(3, 0.5)
        counts = lat.step_mcs(3)
        got, _ = lat.get()
    ref = o.init(1024, 3, 0.5)
    want = o.run(ref, 3.9, 0.5, 3, 0, 3, threads=THREADS)
    assert np.array_equal(counts, want) and np.array_equal(got, ref)


def test_autotuned_schedule_is_used_by_auto(o, pgg):
    """After pgg_autotune the AUTO schedule of every context with that (L, layout) resolves to
    the winner, including kernels whose launch shape is derived at resolution time."""
    L = 1024
    with pgg.Lattice(L, 3.9, 0.5, layout="bitpack") as lat:
        lat.seed(2)
        best = lat.autotune(1)
    with pgg.Lattice(L, 3.9, 0.5, layout="bitpack") as lat:
        assert lat.schedule()["kernel"] == best["kernel"]
        lat.seed(2)
        counts = lat.step_mcs(3)
        got, _ = lat.get()
    ref = o.init(L, 2, 0.5)
    want = o.run(ref, 3.9, 0.5, 2, 0, 3, threads=THREADS)
    assert np.array_equal(counts, want) and np.array_equal(got, ref)
    for kernel in ("resident", "direct"):
        with pgg.Lattice(L, 3.9, 0.5, layout="bitpack") as lat:
            lat.set_schedule(kernel)
            s = lat.schedule()
            assert s["kernel"] == kernel and (kernel != "resident" or s["tile_x"] > 0)


class _DeviceBytes:
    """A raw device buffer as a CUDA array (zero-copy view for torch)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": (n,), "typestr": "|u1", "version": 3}


@pytest.mark.parametrize("layout", ["bitpack", "u8"])
def test_lattice_written_through_device_pointer(o, pgg, layout):
    """A lattice the caller writes through pgg_lattice_device_ptr between resident steps is the one
    the next step advances: the column-class copy the resident kernel keeps between calls belongs
    to the old lattice and must not be reused."""
    import torch
    L = 1024
    with pgg.Lattice(L, 3.9, 0.5, layout=layout) as lat:
        lat.set_schedule("resident")
        lat.seed(5, 0.5)
        lat.step_mcs(2)  # the kernel now keeps the class copy of this lattice
        new = o.init(L, 9, 0.3)
        if layout == "bitpack":
            words = (new.reshape(L, L // 32, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(-1)
            host = words.astype(np.uint32).view(np.uint8).reshape(-1)
        else:
            host = np.ascontiguousarray(new, dtype=np.uint8).reshape(-1)
        ptr, nbytes = lat.device_ptr()
        assert nbytes == host.size
        view = torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")
        view.copy_(torch.from_numpy(host).cuda())  # on the context's (current) stream
        got = lat.step_mcs(3)
        final, step = lat.get()
    want = o.run(new, 3.9, 0.5, 5, 32, 3, threads=THREADS)
    assert step == 80
    assert np.array_equal(got, want)
    assert np.array_equal(final, new)
