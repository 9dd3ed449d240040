"""Host-side sharding of the MI hot path across ranks (one process per GPU).

The path partitions into independent units: scan pairs, or the poses of one batch.
Pairs are spread over ranks with no exchange at all (weak scaling).  When one pose
batch is split, each rank evaluates its contiguous pose range and the ranks agree on
the batch's argmax (Eq. 1) by one max-reduction of a packed (MI, index) key in which
the lower index wins ties -- the only exchange the method has.
"""
from __future__ import annotations

import struct


def shard_range(n: int, rank: int, world: int):
    """Contiguous [start, stop) share of n units for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _orderable(mi: float) -> int:
    u = struct.unpack("<I", struct.pack("<f", mi))[0]
    return (~u & 0xFFFFFFFF) if (u & 0x80000000) else (u | 0x80000000)


def pack_argmax(mi: float, index: int) -> int:
    """Signed 64-bit key whose maximum is the largest FP32 MI, ties to the lowest index."""
    if not (0 <= index < 0xFFFFFFFF):
        raise ValueError("index out of range")
    key = (_orderable(mi) << 32) | (0xFFFFFFFF - index)
    return key - (1 << 63)


def unpack_argmax(key: int) -> int:
    return 0xFFFFFFFF - ((key + (1 << 63)) & 0xFFFFFFFF)


def global_argmax(local_mi: float, local_index: int, group=None) -> int:
    """Batch-wide argmax from each rank's best (MI, global index)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([pack_argmax(local_mi, local_index)], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return unpack_argmax(int(t.item()))


def max_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
