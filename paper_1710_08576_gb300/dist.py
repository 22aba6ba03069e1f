"""Multi-GPU layout of the excision workload: replicas with weak scaling, no data-path collective.

Streams are independent and the digital noise is keyed by (stream id, absolute sample index),
so N GPUs excise N disjoint sets of streams (N antenna sets, Section II-C) with no exchange.
The only collectives are the benchmark's barrier and the reductions of its timing and totals.
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, local_rank, world_size) from the torchrun environment (defaults: one process)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def stream_ids(rank: int, nstreams: int, stride: int = 1000):
    """Stream ids (feed keys and noise stream ids) of rank `rank`: its own antenna set."""
    return [s + stride * rank for s in range(nstreams)]


class Group:
    """Barrier and max/sum reductions over the ranks (a no-op group for one process)."""

    def __init__(self, backend: str | None = None, device=None):
        self.rank, self.local_rank, self.world = env_rank()
        self.dist = None
        self.device = device
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                if backend == "nccl":
                    dist.init_process_group("nccl", device_id=device)
                else:
                    dist.init_process_group(backend or "gloo")
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, v: float, op) -> float:
        if self.dist is None:
            return float(v)
        import torch
        dev = self.device if self.device is not None else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v: float) -> float:
        return self._reduce(v, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, v: float) -> float:
        return self._reduce(v, None if self.dist is None else self.dist.ReduceOp.SUM)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def throughput(units_per_rank: float, seconds_per_rank: float, group: Group) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return group.sum(units_per_rank) / group.max(seconds_per_rank)
