"""Replica bookkeeping for runs with one process per GPU (torchrun).

One real-time iteration does not shard: its stages are sequential and its QP has N nu
variables.  A run on N GPUs therefore steps N independent replicas, one per rank, with no
exchange on the data path; only the timing is combined.  The whole job has done
N x steps instance steps when the slowest rank finishes, so the aggregate rate is
N x 1000 / (max over ranks of the milliseconds per step).  Host logic only (the collective
is a barrier and one max-reduction of a scalar).
"""
from __future__ import annotations

import os


class Replicas:
    """Rank, world size and the two collectives of a replicated run.

    With WORLD_SIZE > 1 the default process group is created with `backend` (nccl on the
    GPUs, gloo for tests on the CPU); `device` holds the reduction's scalar.
    """

    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self._dist = None
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self._dist = dist

    @property
    def leader(self):
        """The rank that reports (rank 0)."""
        return self.rank == 0

    def barrier(self):
        if self._dist is not None:
            self._dist.barrier()

    def max_over_ranks(self, value):
        """The largest value any rank passes (every rank gets it)."""
        if self._dist is None:
            return float(value)
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def steps_per_s(self, ms_per_step):
        """Whole-job instance steps per second from the slowest rank's milliseconds per step."""
        return self.world * 1000.0 / ms_per_step

    def close(self):
        if self._dist is not None and self._dist.is_initialized():
            self._dist.destroy_process_group()
        self._dist = None
