"""Host-side multi-process helpers (one process per GPU).

The contraction shards without any exchange on its data path: bitstring
batches are independent problems, and slices are independent terms of a sum
(App. A, "Slicing": the contractions for the values of the fixed legs can run
in parallel and are added at the end).  So ranks either run their own batches
(weak scaling), or own contiguous blocks of slice ids and add their partial
FP64 amplitudes once at the end.  These helpers work with the gloo backend on
CPU tensors and with NCCL on CUDA tensors.
"""
from __future__ import annotations

import os
from typing import Tuple

import numpy as np


def env_rank_world() -> Tuple[int, int]:
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [lo, hi) of n units owned by `rank` (sizes differ by
    at most one, earlier ranks take the extra units)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _device():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_partial_amplitudes(partial: np.ndarray, world: int) -> np.ndarray:
    """FP64 sum over ranks of per-rank partial amplitudes (complex128 array,
    same bitstrings on every rank): the one exchange step when ranks own
    blocks of slices."""
    partial = np.ascontiguousarray(partial, dtype=np.complex128)
    if world == 1:
        return partial.copy()
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(partial.view(np.float64).copy()).to(_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy().view(np.complex128).copy()
