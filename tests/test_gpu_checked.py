"""The index-checking build of the library (-DPGG_CHECKED=1): every shared- and global-memory
index of the tiled, direct and resident kernels is tested against its buffer before the
access, and a failure is reported through the context's status word (the next synchronising
call raises). These cases run the kernels across lattice sizes, ragged tiles, launch shapes,
both layouts and both games in that build, and require both no failed check and the oracle's
lattice and counts bit for bit. (compute-sanitizer is not available on the GPU pool; this is
its stand-in for out-of-bounds accesses.)
"""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
PD = (1.0, 0.0, 1.04, 0.0)


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


@pytest.fixture(scope="module")
def pgg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1704_08098_gb300 import build, pgg as P
    build.build(checked=True)
    return P


def run_checked(P, o, L, layout, sched, pay, n_mcs, seed, r=3.9, K=0.5):
    ref = o.init(L, seed, 0.5)
    if pay is None:
        want = o.run(ref, r, K, seed, 0, n_mcs, threads=THREADS)
    else:
        want = o.pair_run(ref, pay, K, seed, 0, n_mcs, threads=THREADS)
    with P.Lattice(L, r, K, layout=layout, checked=True) as lat:
        if pay is not None:
            lat.set_game("pairwise", pay)
        lat.set_schedule(**sched)
        lat.seed(seed, 0.5)
        got = lat.step_mcs(n_mcs)
        final, _ = lat.get()   # raises if an index check failed
        assert lat.count() == int(final.sum())
    assert np.array_equal(got, want), (L, layout, sched, pay)
    assert np.array_equal(final, ref), (L, layout, sched, pay)


@pytest.mark.parametrize("game", [None, PD], ids=["group", "pairwise"])
@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L", [256, 768, 1024, 4096])
def test_checked_resident(o, pgg, L, layout, game):
    run_checked(pgg, o, L, layout, dict(kernel="resident"), game, 3 if L < 4096 else 1, 11 + L)


@pytest.mark.parametrize("game", [None, PD], ids=["group", "pairwise"])
@pytest.mark.parametrize("upt,block", [(4, 64), (8, 128), (4, 256)])
@pytest.mark.parametrize("L", [256, 768])
def test_checked_direct(o, pgg, L, upt, block, game):
    run_checked(pgg, o, L, "bitpack", dict(kernel="direct", tile_x=upt, tile_y=block), game, 3, 21 + L)


@pytest.mark.parametrize("game", [None, PD], ids=["group", "pairwise"])
@pytest.mark.parametrize("layout", ["bitpack", "u8"])
@pytest.mark.parametrize("L,tx,ty,k", [(64, 64, 64, 1), (192, 128, 36, 4), (320, 256, 100, 8),
                                        (128, 64, 124, 16), (256, 192, 60, 2)])
def test_checked_tiled(o, pgg, L, tx, ty, k, layout, game):
    run_checked(pgg, o, L, layout, dict(kernel="tiled", steps_per_launch=k, tile_x=tx, tile_y=ty), game, 3,
                31 + L)
