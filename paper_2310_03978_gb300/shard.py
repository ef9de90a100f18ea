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


def contract_resumable(plan, slice_begin: int, slice_end: int, checkpoint: str,
                       chunk: int = 0, on_chunk=None):
    """Contract slices [slice_begin, slice_end) in chunks, keeping a checkpoint of the partial FP64
    amplitudes and of the next slice to contract, so that a job interrupted between chunks
    resumes where it stopped (slices are independent sub-tasks whose results are summed,
    Sec. 3.2 and Sec. 5).

    ``plan`` needs ``contract_host(b, e)`` (the sum over slices [b, e) as a host complex128
    array) and ``info()["slices_in_flight"]``; ``chunk`` is the number of slices per chunk (0: the
    plan's slices in flight).  Chunk results are added in FP64 in chunk order.  The checkpoint
    (numpy .npz: amplitudes, next slice, range) is written to a temporary name and renamed, so
    the file on disk is always complete; a checkpoint for another slice range is rejected.
    ``on_chunk(next_slice)`` runs after each saved chunk.  Returns the amplitudes of the range."""
    import os
    import numpy as np
    if slice_end <= slice_begin:
        raise ValueError("empty slice range")
    if chunk <= 0:
        chunk = max(1, int(plan.info()["slices_in_flight"]))
    nxt, amps = slice_begin, None
    if os.path.exists(checkpoint):
        with np.load(checkpoint) as z:
            if int(z["slice_begin"]) != slice_begin or int(z["slice_end"]) != slice_end:
                raise ValueError("checkpoint %s is for slices [%d, %d), not [%d, %d)" % (
                    checkpoint, int(z["slice_begin"]), int(z["slice_end"]), slice_begin,
                    slice_end))
            nxt = int(z["next_slice"])
            amps = np.array(z["amps"], dtype=np.complex128)
    while nxt < slice_end:
        e = min(slice_end, nxt + chunk)
        part = np.asarray(plan.contract_host(nxt, e), dtype=np.complex128)
        amps = part.copy() if amps is None else amps + part
        nxt = e
        tmp = checkpoint + ".tmp.npz"
        np.savez(tmp, amps=amps, next_slice=nxt, slice_begin=slice_begin, slice_end=slice_end)
        os.replace(tmp, checkpoint)
        if on_chunk is not None:
            on_chunk(nxt)
    return amps
