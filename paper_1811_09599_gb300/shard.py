"""Work partitioning across ranks (one process per GPU).

Methods, "Cutting indexes": the paths of one amplitude batch are
independent, and so are bitstrings.  Two partitions follow:

* by bitstrings (weak scaling): every rank contracts its own bitstrings
  with all paths; nothing is exchanged on the data path, only the timing
  is reduced (max over ranks).
* by slices (strong scaling of one batch): the slice range (or a list of
  slice ids, such as the paths that do not vanish identically) is split
  into contiguous shards; each rank sums its shard's contributions and one
  collective, an FP64 sum over ranks of the n_bs x 2^|tile| partial
  amplitudes, completes the batch (the sum over paths is exact up to the
  order of FP64 additions).

The collectives go through torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Callable, Sequence, Tuple, Union

import torch
import torch.distributed as dist


def shard(total: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) share of `total` units for `rank` of `world`; the
    first total % world ranks take one extra unit."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def bitstring_seed(base: int, rank: int) -> int:
    """Seed of a rank's own bitstrings under the bitstring partition."""
    return base + rank


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest `value` over all ranks (timings are reduced this way)."""
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def slice_sharded_amplitudes(compute: Callable[[Sequence[int]], torch.Tensor],
                             slices: Union[int, Sequence[int]], group=None) -> torch.Tensor:
    """Sum over paths, split across ranks: `slices` is the number of slices
    (all ids 0..P-1) or a list of slice ids, e.g. the paths that do not
    vanish identically (Plan.nonzero_slices), so that every rank gets an
    equal share of the paths that cost work.  compute(slice_ids) returns
    this rank's partial complex128 amplitudes (zeros for an empty list); the
    partial sums are added over ranks in FP64 and every rank gets the
    total."""
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    ids = list(range(slices)) if isinstance(slices, int) else [int(s) for s in slices]
    lo, hi = shard(len(ids), rank, world)
    part = compute(ids[lo:hi])
    if part.dtype != torch.complex128:
        raise TypeError("partial amplitudes must be complex128")
    if world > 1:
        flat = torch.view_as_real(part.contiguous())
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        part = torch.view_as_complex(flat)
    return part
