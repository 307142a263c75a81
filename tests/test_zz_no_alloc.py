"""pgg_step_mcs_noalloc, the entry point for callers that cannot allocate device memory (plug-ins
whose host application owns all device memory, services that must not allocate after start-up),
checked over two calls in a row against the CPU oracle and against the context-based
pgg_step_mcs on the same inputs: lattices and per-MCS counts are exact results, so every
comparison is exact equality.

Kept in a file of its own that pytest collects last."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_1704_08098_gb300 import build, pgg
    build.build()
    return torch, pgg


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


def to_device_layout(torch, host_lat, layout):
    if layout == "u8":
        return torch.from_numpy(np.ascontiguousarray(host_lat)).cuda()
    bits = np.packbits(host_lat.astype(np.uint8), axis=1, bitorder="little")
    return torch.from_numpy(np.ascontiguousarray(bits)).cuda()


def from_device_layout(torch, dev, L, layout):
    a = dev.cpu().numpy()
    if layout == "u8":
        return a.reshape(L, L)
    return np.unpackbits(a.reshape(L, L // 8), axis=1, bitorder="little")


# L = 1088 leaves a partial tile in both directions (tiles of 1024 x 128 sites); L = 2048 (uint8)
# and L = 4096 (bit-packed) fill the 4 MiB scratch lattice exactly.
@pytest.mark.parametrize("layout,L,n", [("u8", 256, 6), ("bitpack", 512, 6), ("bitpack", 64, 6),
                                        ("u8", 1088, 3), ("bitpack", 1088, 3),
                                        ("u8", 2048, 2), ("bitpack", 4096, 2)])
def test_noalloc_matches_oracle_twice(env, o, layout, L, n):
    torch, pgg = env
    r, K, seed = 3.8, 0.5, 23
    ref = o.init(L, seed, 0.5)
    dev_in = to_device_layout(torch, ref, layout)
    dev_out = torch.empty_like(dev_in)
    counts = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    # first call: separate input and output buffers, from step 0
    pgg.step_mcs_noalloc(dev_in.data_ptr(), dev_out.data_ptr(), L, layout, r, K, seed, 0, n,
                         counts.data_ptr())
    want = o.run(ref, r, K, seed, 0, n, threads=THREADS)
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(from_device_layout(torch, dev_out, L, layout), ref)
    # the input buffer is left as it was
    assert np.array_equal(from_device_layout(torch, dev_in, L, layout), o.init(L, seed, 0.5))
    # second call: in place, continuing from the returned state; the scratch array still holds
    # the first call's intermediate lattice and must not leak into this one
    counts.fill_(-1)
    pgg.step_mcs_noalloc(dev_out.data_ptr(), dev_out.data_ptr(), L, layout, r, K, seed, 16 * n, n,
                         counts.data_ptr())
    want = o.run(ref, r, K, seed, 16 * n, n, threads=THREADS)
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(from_device_layout(torch, dev_out, L, layout), ref)


@pytest.mark.parametrize("layout,L", [("u8", 256), ("bitpack", 512), ("bitpack", 64)])
def test_noalloc_matches_context_path_twice(env, layout, L):
    torch, pgg = env
    r, K, seed = 3.8, 0.5, 17
    with pgg.Lattice(L, r, K, layout=layout) as ref:
        ref.seed(seed, 0.5)
        start, step = ref.get()
        dev_in = to_device_layout(torch, start, layout)
        dev_out = torch.empty_like(dev_in)
        counts = torch.zeros(6, dtype=torch.int64, device="cuda")
        # first call: separate input and output buffers
        pgg.step_mcs_noalloc(dev_in.data_ptr(), dev_out.data_ptr(), L, layout, r, K, seed, step,
                             6, counts.data_ptr())
        want_counts = ref.step_mcs(6)
        want_lat, want_step = ref.get()
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().astype(np.uint64), want_counts)
        assert np.array_equal(from_device_layout(torch, dev_out, L, layout), want_lat)
        # second call: in place, continuing from the returned state
        pgg.step_mcs_noalloc(dev_out.data_ptr(), dev_out.data_ptr(), L, layout, r, K, seed,
                             want_step, 6, counts.data_ptr())
        want_counts = ref.step_mcs(6)
        want_lat, _ = ref.get()
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy().astype(np.uint64), want_counts)
        assert np.array_equal(from_device_layout(torch, dev_out, L, layout), want_lat)


def test_noalloc_rejects_bad_arguments(env):
    torch, pgg = env
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pgg.PGGError) as exc:
        pgg.step_mcs_noalloc(buf.data_ptr(), buf.data_ptr(), 8192, "bitpack", 4.0, 0.5, 1, 0, 1)
    assert exc.value.status == pgg.PGG_ERR_ARG and "scratch" in str(exc.value)
    with pytest.raises(pgg.PGGError):
        pgg.step_mcs_noalloc(buf.data_ptr(), buf.data_ptr(), 4096, "u8", 4.0, 0.5, 1, 0, 1)
    # step counters that would pass 2^56, including counts whose 16 n_mcs wraps a uint64
    for step0, n in ((2 ** 56 - 16, 1), (2 ** 56, 0), (0, 2 ** 60), (5, 2 ** 62)):
        with pytest.raises(pgg.PGGError) as exc:
            pgg.step_mcs_noalloc(buf.data_ptr(), buf.data_ptr(), 64, "bitpack", 4.0, 0.5, 1, step0, n)
        assert exc.value.status == pgg.PGG_ERR_ARG and "2^56" in str(exc.value)
