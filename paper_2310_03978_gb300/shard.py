"""Multi-GPU sharding of the sliced contraction (host logic; one process per GPU).

Slices are independent sub-tasks whose results are summed (Sec. 3.2; Sec. 5: each GPU ran part of
the sub-tasks and the final outcome was the sum of the resulting tensors).  Two ways to shard:

* weak scaling: every rank contracts its own batch of 2^k amplitudes (the same circuit with its
  own seeded closed bits, hence the same network structure, path and work) and nothing is
  exchanged;
* strong scaling: the ranks split one batch's slices into contiguous ranges, each accumulates its
  partial amplitudes in FP64, and one sum-reduce of the 2^k complex128 vector combines them.

The functions take a torch.distributed process group (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from . import workload as W


def rank_network(wl, rank: int):
    """Network of rank `rank` for weak scaling: the workload's circuit with rank-specific seeded
    closed bits (rank 0 keeps the workload's own).  Labels, path and slices are unchanged."""
    if rank == 0:
        return wl.network
    net = wl.network
    rng = W.Xoshiro256ss(W.BASE_SEED + 1 + 7919 * rank)
    closed = {q: rng.below(2) for q in net.closed_bits}
    return W.build_network(wl.circuit, net.open_qubits, closed)


def slice_range(num_slices: int, rank: int, world: int):
    """Contiguous slice range [begin, end) of `rank` for strong scaling; the ranges of all ranks
    partition [0, num_slices) and differ in length by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(num_slices, world)
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    return begin, end


def reduce_amplitudes(amps, group=None):
    """Sum the ranks' partial amplitude vectors (complex128 tensors, in place) in FP64."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return amps
    view = torch.view_as_real(amps)
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return amps


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Largest value over ranks (the bench's step time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
