"""One lattice split into row bands over gloo ranks on CPU.

Each rank updates the sublattice sites of its own rows with the oracle's elementary update and,
after every sublattice step, refreshes its 3 halo rows above and below from the neighbouring
ranks (point-to-point send/receive): the decomposition the resident kernel uses across SMs, and
the one a lattice spread over several GPUs would use. Sites of one step are at least 4 apart and
an update reads 3 rows either side (Section IV), so a step needs the halo only as it was after
the previous step; every draw is keyed by (seed, step, site), so the banded run must reproduce
the single-process oracle bit for bit, with the count after each MCS summed over the ranks by an
all-reduce.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = 3  # halo rows: the read radius of the group game


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def band(rank, world, L):
    return rank * L // world, (rank + 1) * L // world


def _worker(rank, world, port, L, r, K, seed, n_mcs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle as orc
    o = orc.Oracle()
    lat = o.init(L, seed, 0.5)  # every rank starts from the same state and trusts its band + halo only
    r0, r1 = band(rank, world, L)
    up, down = (rank - 1) % world, (rank + 1) % world
    counts = []
    for k in range(16 * n_mcs):
        off = o.offset(seed, k)
        oi, oj = off >> 2, off & 3
        for i in range(r0 + ((oi - r0) & 3), r1, 4):
            for j in range(oj, L, 4):
                a, b = i >> 2, j >> 2
                o.elementary_update(lat, i, j, o.dir(seed, k, a, b), o.u(seed, k, a, b), r, K)
        # the band's first H rows are the upper neighbour's lower halo, its last H rows the lower
        # neighbour's upper halo
        top = torch.from_numpy(lat[r0:r0 + H].copy())
        bot = torch.from_numpy(lat[r1 - H:r1].copy())
        from_up, from_down = torch.empty_like(top), torch.empty_like(bot)
        reqs = [dist.isend(top, up, tag=2 * k), dist.isend(bot, down, tag=2 * k + 1),
                dist.irecv(from_up, up, tag=2 * k + 1), dist.irecv(from_down, down, tag=2 * k)]
        for q in reqs:
            q.wait()
        lat[[(r0 - H + t) % L for t in range(H)]] = from_up.numpy()
        lat[[(r1 + t) % L for t in range(H)]] = from_down.numpy()
        if k % 16 == 15:
            c = torch.tensor([int(lat[r0:r1].sum())], dtype=torch.int64)
            dist.all_reduce(c)
            counts.append(int(c.item()))
    out.put((rank, r0, r1, lat[r0:r1].copy(), counts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,L,r,K,seed,n_mcs", [(2, 32, 3.9, 0.5, 11, 12), (3, 48, 4.4, 0.3, 12, 8)])
def test_banded_run_with_halo_exchange_matches_oracle(world, L, r, K, seed, n_mcs):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(rk, world, port, L, r, K, seed, n_mcs, q))
             for rk in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    o = oracle.Oracle()
    ref = o.init(L, seed, 0.5)
    want = o.run(ref, r, K, seed, 0, n_mcs)
    got = np.zeros_like(ref)
    for rank, r0, r1, rows, counts in parts:
        got[r0:r1] = rows
        assert counts == [int(c) for c in want], rank
    assert np.array_equal(got, ref)
    assert int(want[-1]) != int(o.init(L, seed, 0.5).sum())  # the run did change the lattice
