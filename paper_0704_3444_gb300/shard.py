"""Independent simulations split across the ranks of a process group, by bytes.

Instances of a batch (the paper's sweeps of Sec. 4, or any set of unrelated problems)
exchange nothing, so across several GPUs each rank simply advances its own share in its
own ``Batch``; no collective is needed on the data path.  A step of a share takes about
as long as its instances' stored distributions take to cross HBM (every value read once
and written once per step), so the shares are balanced by those bytes: each instance,
largest first, goes to the rank with the fewest bytes so far (ties to the lower rank).
The split is deterministic, and the most and least loaded ranks differ by at most the
bytes of one instance (when the most loaded rank took its last instance it was the least
loaded).
"""
from __future__ import annotations

from typing import List, Sequence

__all__ = ["instance_bytes", "partition_by_bytes", "share"]

_Q = {"d2q9": 9, "d1q3": 3, "d3q19": 19}
_STORAGE = {"fp64": 72 // 9, "fp32": 4, "bf16": 2, "fp16": 2}


def instance_bytes(p, precision: str = "fp32") -> int:
    """Bytes one timestep of problem ``p`` moves at least: its q N stored values per site
    read and written once (16-bit formats: plus the FP32 reference density per site and
    component)."""
    q = _Q[getattr(p, "lattice", "d2q9")]
    per = q * _STORAGE[precision] + (4 if precision in ("bf16", "fp16") else 0)
    return 2 * p.ncomp * p.nx * p.ny * max(int(getattr(p, "nz", 1)), 1) * per


def partition_by_bytes(problems: Sequence, world: int, precision: str = "fp32") -> List[List[int]]:
    """Indices of the instances each of ``world`` ranks advances (each list ascending)."""
    if world < 1:
        raise ValueError("world >= 1")
    sizes = [instance_bytes(p, precision) for p in problems]
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(k)
        load[r] += sizes[k]
    return [sorted(p) for p in parts]


def share(problems: Sequence, rank: int, world: int, precision: str = "fp32") -> List[int]:
    """Indices of the instances rank ``rank`` of ``world`` advances."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside 0..{world - 1}")
    return partition_by_bytes(problems, world, precision)[rank]
