"""Multi-rank sharding on CPU: world size 2 over gloo, one spawned process per rank.

Strong scaling: each rank contracts its contiguous slice range (here with the CPU oracle) and the
single FP64 sum-reduce of the amplitude vectors must give the whole contraction.  Weak scaling:
every rank's network has the same structure and path and its own closed bits.
"""
import os
import socket

import numpy as np
import pytest

from paper_2310_03978_gb300 import shard
from paper_2310_03978_gb300 import workload as W

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.small_workload()
        net = wl.network
        sliced = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
        b, e = shard.slice_range(1 << len(sliced), rank, world)
        amps = torch.from_numpy(O.contract_network(net, wl.path, sliced, b, e).copy())
        shard.reduce_amplitudes(amps)
        t = shard.max_over_ranks(0.5 + rank)
        mine = shard.rank_network(wl, rank)
        weak = O.contract_network(mine, wl.path)
        np.save(os.path.join(out_dir, "strong_%d.npy" % rank), amps.numpy())
        np.save(os.path.join(out_dir, "weak_%d.npy" % rank), weak)
        with open(os.path.join(out_dir, "meta_%d.txt" % rank), "w") as f:
            f.write("%r\n%r\n%r\n" % (t, (b, e), sorted(mine.closed_bits.items())))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    import torch.multiprocessing as mp
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True,
                       start_method="spawn")
    return out


def test_strong_scaling_sum_reduce_gives_the_whole_contraction(two_ranks):
    from oracle import oracle as O
    wl = W.small_workload()
    full = O.contract_network(wl.network, wl.path)
    for r in range(2):
        got = np.load(os.path.join(two_ranks, "strong_%d.npy" % r))
        np.testing.assert_allclose(got, full, rtol=0, atol=1e-13)


def test_ranks_agree_on_max_time_and_split_the_slices(two_ranks):
    metas = [open(os.path.join(two_ranks, "meta_%d.txt" % r)).read().splitlines()
             for r in range(2)]
    assert float(metas[0][0]) == float(metas[1][0]) == 1.5
    assert eval(metas[0][1]) == (0, 4) and eval(metas[1][1]) == (4, 8)


def test_weak_scaling_ranks_have_own_closed_bits_same_structure(two_ranks):
    from oracle import oracle as O
    wl = W.small_workload()
    r1 = shard.rank_network(wl, 1)
    assert r1.labels == wl.network.labels and r1.open_labels == wl.network.open_labels
    assert r1.closed_bits != wl.network.closed_bits
    w0 = np.load(os.path.join(two_ranks, "weak_0.npy"))
    w1 = np.load(os.path.join(two_ranks, "weak_1.npy"))
    np.testing.assert_allclose(w0, O.contract_network(wl.network, wl.path), atol=1e-13)
    np.testing.assert_allclose(w1, O.contract_network(r1, wl.path), atol=1e-13)
    assert np.abs(w0 - w1).max() > 1e-6


@pytest.mark.parametrize("num,world", [(16, 1), (16, 2), (16, 3), (7, 4), (3, 8), (65536, 6)])
def test_slice_ranges_partition(num, world):
    ranges = [shard.slice_range(num, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == num
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1
    lens = [e - b for b, e in ranges]
    assert max(lens) - min(lens) <= 1


class _OraclePlan:
    """Stand-in for a plan on the CPU: contract_host sums the oracle's slices [b, e)."""

    def __init__(self, wl, sliced, in_flight=2):
        from oracle import oracle as O
        self.O, self.wl, self.sliced, self.in_flight = O, wl, sliced, in_flight
        self.calls = []

    def info(self):
        return {"slices_in_flight": self.in_flight, "num_slices": 1 << len(self.sliced)}

    def contract_host(self, b, e):
        self.calls.append((b, e))
        return self.O.contract_network(self.wl.network, self.wl.path, self.sliced, b, e)


def test_checkpointed_slice_range_resumes_after_interruption(tmp_path):
    from oracle import oracle as O
    wl = W.small_workload()
    net = wl.network
    sliced = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    full = O.contract_network(net, wl.path)
    ck = str(tmp_path / "ck.npz")

    class Stop(Exception):
        pass

    def stop_after_two(nxt):
        if nxt >= 4:
            raise Stop()

    plan = _OraclePlan(wl, sliced)
    with pytest.raises(Stop):
        shard.contract_resumable(plan, 0, 8, ck, on_chunk=stop_after_two)
    assert plan.calls == [(0, 2), (2, 4)]
    # a new process resumes at slice 4 and finishes the range
    plan2 = _OraclePlan(wl, sliced)
    amps = shard.contract_resumable(plan2, 0, 8, ck)
    assert plan2.calls == [(4, 6), (6, 8)]
    np.testing.assert_allclose(amps, full, rtol=0, atol=1e-13)
    # finished: nothing left to do; another range is refused
    plan3 = _OraclePlan(wl, sliced)
    np.testing.assert_allclose(shard.contract_resumable(plan3, 0, 8, ck), full, atol=1e-13)
    assert plan3.calls == []
    with pytest.raises(ValueError):
        shard.contract_resumable(plan3, 0, 4, ck)
