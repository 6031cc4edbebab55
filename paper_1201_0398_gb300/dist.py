"""Rank setup and timing reductions for multi-process runs (one process per GPU).

ECB blocks are independent (Section 3: no dependency between the pixels), so
ranks shard the work with no data-path collective: each rank enciphers its own
buffers (weak scaling).  The process group carries only the barrier around the
timed region and the max-over-ranks of the elapsed time.  Works with NCCL on
GPUs and with gloo on CPUs (the tests run it as two gloo ranks).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Ranks:
    world: int
    rank: int
    local: int
    backend: str | None

    @property
    def distributed(self) -> bool:
        return self.world > 1


def setup(backend: str | None = None) -> Ranks:
    """Reads RANK/LOCAL_RANK/WORLD_SIZE (torchrun); initialises the process group
    when WORLD_SIZE > 1 (NCCL if CUDA is available, else gloo)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return Ranks(1, 0, 0, None)
    import torch
    import torch.distributed as dist

    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if not dist.is_initialized():
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return Ranks(world, rank, local, backend)


def barrier(r: Ranks) -> None:
    if r.distributed:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(r: Ranks, value: float) -> float:
    """The largest value any rank passes (each rank's elapsed time -> the job's)."""
    if not r.distributed:
        return value
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if r.backend == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_seed(base_seed: int, r: Ranks) -> int:
    """Seed of this rank's shard: distinct data per rank, the same key schedule."""
    return base_seed + 97 * r.rank


def teardown(r: Ranks) -> None:
    if r.distributed:
        import torch.distributed as dist

        if dist.is_initialized():
            dist.destroy_process_group()
