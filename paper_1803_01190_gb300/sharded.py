"""i-partition of the Eq. 1-2 force sum over the ranks of a process group.

The paper divides the N particles into k contiguous blocks, one per GPU
(section 2, Figs. 1-3): every GPU holds all positions and computes the forces
on its own N/k particles.  Here rank r owns the particles
[offsets[r], offsets[r] + counts[r]); one force evaluation is

  1. one all-gather of every rank's packed (x, y, z, m) rows into each rank's
     own device memory (torch.distributed: NCCL between GPUs, gloo on CPU),
  2. the rank's own rows against all N on its GPU (nbody_accel_rows: the
     one-sided kernels, so the rows equal those of a single-GPU evaluation with
     the each-pair-once path off, bit for bit).

The exchange is the only collective; the gathered positions land in local
memory before any kernel reads them (no peer or multicast loads).  This module
only moves arrays and calls the C ABI; the arithmetic runs in the library's
kernels.  `local_force` replaces step 2 with another function of the same
signature (the CPU tests use it to check the partition and the gather against
the oracle without a GPU).
"""
import numpy as np


def partition(n, world):
    """Contiguous blocks of as equal size as possible: (counts, offsets)."""
    base, extra = divmod(int(n), int(world))
    counts = [base + (1 if r < extra else 0) for r in range(world)]
    offsets = [0]
    for c in counts[:-1]:
        offsets.append(offsets[-1] + c)
    return counts, offsets


class ShardedForce:
    """Eq. 1-2 on an i-partition of n particles over the ranks of `group`.

    mode, eps, G: as for Simulation.  device: where the gathered arrays live
    ("cuda" for the GPU path).  local_force(pos_all, mass_all, i0, ni) ->
    (acc (ni,3), pot (ni,)) overrides the GPU rows call."""

    def __init__(self, n, mode="fp64", eps=0.01, G=1.0, group=None, device="cuda",
                 local_force=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.n = int(n)
        self.counts, self.offsets = partition(self.n, self.world)
        self.cmax = max(self.counts)
        self.device = device
        self.local_force = local_force
        self.sim = None
        if local_force is None:
            from . import Simulation
            self.sim = Simulation(self.n, mode=mode, eps=eps, G=G)

    @property
    def rows(self):
        """(i0, ni) of this rank."""
        return self.offsets[self.rank], self.counts[self.rank]

    def gather(self, pos_local, mass_local):
        """All ranks' (pos, mass) rows, in particle order, on this rank's device."""
        t = self.torch
        i0, ni = self.rows
        packed = t.zeros((self.cmax, 4), dtype=t.float64, device=self.device)
        if ni:
            packed[:ni, :3] = t.as_tensor(pos_local, dtype=t.float64, device=self.device).reshape(ni, 3)
            packed[:ni, 3] = t.as_tensor(mass_local, dtype=t.float64, device=self.device).reshape(ni)
        parts = [t.empty_like(packed) for _ in range(self.world)]
        self.dist.all_gather(parts, packed, group=self.group)
        full = t.cat([parts[r][:self.counts[r]] for r in range(self.world)])
        return full[:, :3].contiguous(), full[:, 3].contiguous()

    def accel(self, pos_local, mass_local):
        """Accelerations and potentials of this rank's own particles."""
        pos_all, mass_all = self.gather(pos_local, mass_local)
        i0, ni = self.rows
        if ni == 0:
            return np.empty((0, 3)), np.empty(0)
        if self.local_force is not None:
            return self.local_force(pos_all, mass_all, i0, ni)
        return self.sim.accel_rows(i0, ni, pos_all, mass_all)

    def close(self):
        if self.sim is not None:
            self.sim.close()
            self.sim = None
