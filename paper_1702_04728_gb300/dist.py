"""Multi-GPU layout of the fan-beam path: channels shard across ranks.

Frequency channels are independent (the paper runs the pipeline per channel,
one channel per GPU, Sec. 2), so N ranks process N disjoint channel sets with
no exchange on the data path; the only collective is the max-over-ranks
reduction of the step time.
"""
from __future__ import annotations

from typing import List

CHAN_BW_HZ = 390625.0
NODE_SLICE_HZ = (410e6, 520e6, 650e6, 790e6)


def rank_channels(rank: int, world: int, base=NODE_SLICE_HZ) -> List[float]:
    """Channel centre frequencies of rank ``rank``: the node slice shifted by
    ``rank`` coarse channels, so ranks hold disjoint channels of the band."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return [f + rank * CHAN_BW_HZ for f in base]


def rank_seed(rank: int, seed: int = 0) -> int:
    return seed + 1000 * rank


def max_over_ranks(values, group=None):
    """Element-wise max of a list of floats over all ranks (any backend)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.cpu().tolist()
