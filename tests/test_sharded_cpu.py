"""The i-partition of the force sum (the paper's N/k split, section 2) on CPU:
gloo process groups of 2 and 3 ranks, each rank owning a contiguous block of
particles, one all-gather of the packed positions and masses, then its own
rows against all N.  The per-rank force is the oracle (rows mode) here, so
the test checks the partition and the exchange: the ranks' rows, put back
together, must equal the single-process oracle bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1803_01190_gb300.sharded import partition  # noqa: E402


def test_partition_covers_every_particle_once():
    for n, k in ((10, 3), (1001, 2), (1, 2), (4096, 8), (7, 7)):
        counts, offsets = partition(n, k)
        assert sum(counts) == n and len(counts) == k
        assert max(counts) - min(counts) <= 1
        assert offsets == list(np.cumsum([0] + counts[:-1]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import nbody_ics
    import oracle
    from paper_1803_01190_gb300.sharded import ShardedForce
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = nbody_ics.workload("sweep_plummer", n=n)

    def oracle_rows(pos_all, mass_all, i0, ni):
        a, p, _ = oracle.accel(pos_all.numpy(), mass_all.numpy(), w["eps"], 0.9,
                               rows=np.arange(i0, i0 + ni), threads=1)
        return a, p

    sf = ShardedForce(n, eps=w["eps"], G=0.9, device="cpu", local_force=oracle_rows)
    i0, ni = sf.rows
    acc, pot = sf.accel(w["pos"][i0:i0 + ni], w["mass"][i0:i0 + ni])
    # put the rows back together on every rank (a test-side gather)
    gathered = [None] * world
    dist.all_gather_object(gathered, (i0, np.asarray(acc), np.asarray(pot)))
    dist.destroy_process_group()
    q.put((rank, gathered))


@pytest.mark.parametrize("world,n", [(2, 1001), (3, 640), (3, 2)])
def test_sharded_rows_equal_single_process(world, n):
    import torch.multiprocessing as mp
    import nbody_ics
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    w = nbody_ics.workload("sweep_plummer", n=n)
    acc_o, pot_o, _ = oracle.accel(w["pos"], w["mass"], w["eps"], 0.9)
    for rank in range(world):
        parts = sorted(res[rank], key=lambda t: t[0])
        acc = np.concatenate([a for _, a, _ in parts])
        pot = np.concatenate([p for _, _, p in parts])
        assert np.array_equal(acc, acc_o) and np.array_equal(pot, pot_o)
