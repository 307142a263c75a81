"""pgg_step_mcs_noalloc, the entry point for callers that cannot allocate device memory
(graph-capture regions, host callbacks, applications that own all device memory), against
the context-based pgg_step_mcs on the same inputs, over two calls in a row.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_1704_08098_gb300 import build, pgg
    build.build()
    return torch, pgg


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


def test_noalloc_rejects_oversized_lattices(env):
    torch, pgg = env
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pgg.PGGError) as exc:
        pgg.step_mcs_noalloc(buf.data_ptr(), buf.data_ptr(), 8192, "bitpack", 4.0, 0.5, 1, 0, 1)
    assert exc.value.status == pgg.PGG_ERR_ARG and "scratch" in str(exc.value)
    with pytest.raises(pgg.PGGError):
        pgg.step_mcs_noalloc(buf.data_ptr(), buf.data_ptr(), 4096, "u8", 4.0, 0.5, 1, 0, 1)
