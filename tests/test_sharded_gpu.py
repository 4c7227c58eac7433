"""The per-GPU share of the i-partitioned force sum (nbody_accel_rows) on one
GPU: k row blocks evaluated one after another reproduce, bit for bit, the
rows of one full evaluation with the same kernels (each-pair-once path off,
input order), in every precision mode, and the FP64 rows pass the parity gate
against the oracle.  The sharded driver runs once as a one-rank NCCL group."""
import os
import socket

import numpy as np
import pytest

import nbody_ics
import oracle
from tests.gates import fp64_accel_gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as m
    return m


@pytest.mark.parametrize("mode", ["fp64", "mixed", "f64e", "fp32"])
def test_row_blocks_equal_full_evaluation(nb, mode):
    from paper_1803_01190_gb300.sharded import partition
    n = 40000 + 37
    w = nbody_ics.workload("sweep_plummer", n=n)
    with nb.Simulation(n, mode, eps=w["eps"]) as sim:
        if mode in ("fp64", "f64e"):
            sim.set_symmetric(0)
        if mode != "fp32":
            sim.set_order("input")
        a_full, p_full = sim.accel(w["pos"], w["mass"])
        counts, offsets = partition(n, 3)
        rows = [sim.accel_rows(i0, ni, w["pos"], w["mass"]) for i0, ni in zip(offsets, counts)]
        with pytest.raises(nb.NbodyError):
            sim.accel_rows(n - 5, 6, w["pos"], w["mass"])
    a = np.concatenate([r[0] for r in rows])
    p = np.concatenate([r[1] for r in rows])
    assert np.array_equal(a, a_full) and np.array_equal(p, p_full)
    if mode == "fp64":
        r = np.sort(np.random.default_rng(1).choice(n, 256, replace=False))
        acc_o, pot_o, smag = oracle.accel(w["pos"], w["mass"], w["eps"], rows=r)
        assert fp64_accel_gate(a[r], acc_o, smag, n)[0].all()
        assert np.all(np.abs(p[r] - pot_o) <= 1e-12 * np.abs(pot_o))


def test_sharded_force_one_rank_nccl(nb):
    import torch
    import torch.distributed as dist
    from paper_1803_01190_gb300.sharded import ShardedForce
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        n = 5003
        w = nbody_ics.workload("sweep_uniform", n=n)
        sf = ShardedForce(n, mode="fp64", eps=w["eps"])
        acc, pot = sf.accel(torch.tensor(w["pos"], device="cuda"), torch.tensor(w["mass"], device="cuda"))
        sf.close()
        with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
            a_full, p_full = sim.accel(w["pos"], w["mass"])
        assert np.array_equal(acc.cpu().numpy(), a_full) and np.array_equal(pot.cpu().numpy(), p_full)
    finally:
        dist.destroy_process_group()
