"""Host path optimisation (tn_path_optimize, Sec. 3.2): simulated annealing over the contraction
tree with the three-descendant local update and dynamic slicing.  Pinned against exhaustive
enumeration of all contraction trees of small networks, the Python path replay, path
independence of the oracle's amplitudes, and the argument checks (no GPU needed)."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_03978_gb300 import tn as T
from paper_2310_03978_gb300 import workload as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return T.lib()


def random_network(rng, n, extra_edges, n_open):
    """Connected random graph of n tensors: a random spanning tree plus extra edges (each edge a
    label on its two tensors), and n_open open labels on random tensors."""
    labels = [[] for _ in range(n)]
    nxt = 0
    order = list(rng.permutation(n))
    for i in range(1, n):
        a, b = order[i], order[int(rng.integers(0, i))]
        labels[a].append(nxt)
        labels[b].append(nxt)
        nxt += 1
    for _ in range(extra_edges):
        a, b = rng.choice(n, size=2, replace=False)
        labels[a].append(nxt)
        labels[b].append(nxt)
        nxt += 1
    open_labels = []
    for _ in range(n_open):
        a = int(rng.integers(0, n))
        labels[a].append(nxt)
        open_labels.append(nxt)
        nxt += 1
    return labels, open_labels


def trees(items):
    """Every unordered binary tree over the tuple of leaves ``items``."""
    if len(items) == 1:
        yield items[0]
        return
    first, rest = items[0], items[1:]
    for r in range(0, len(rest)):
        for comb in itertools.combinations(rest, r):
            left = (first,) + comb
            right = tuple(x for x in rest if x not in comb)
            for tl in trees(left):
                for tr in trees(right):
                    yield (tl, tr)


def tree_tcc(tree, sets):
    """T_cc of a tree: 8 real flops per multiply-add, 2^|union| multiply-adds per pair (every
    label on two tensors or open, all dims 2).  Returns (labels of the result, T_cc)."""
    if not isinstance(tree, tuple):
        return sets[tree], 0
    la, ca = tree_tcc(tree[0], sets)
    lb, cb = tree_tcc(tree[1], sets)
    return la ^ lb, ca + cb + 8 * 2 ** len(la | lb)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_annealing_reaches_the_exhaustive_optimum_on_small_networks(seed):
    rng = np.random.default_rng(seed)
    n = 7
    labels, open_labels = random_network(rng, n, 5, 2)
    sets = [frozenset(l) for l in labels]
    best = min(tree_tcc(t, sets)[1] for t in trees(tuple(range(n))))
    start = W.greedy_path(labels, open_labels)
    path, sliced, info = T.path_optimize(labels, open_labels, start, seed=seed, sweeps=400,
                                         sweeps_final=0, t_start=2.0, t_end=0.01, chains=4)
    assert sliced == []
    _, tcc, _ = W.path_cost(labels, open_labels, path)
    assert tcc == best
    assert abs(info["log2_tcc"] - math.log2(best)) < 1e-9


def test_reported_costs_match_the_python_replay_and_improve_on_greedy():
    wl = W.bench_workload()
    net = wl.network
    _, tcc0, _ = W.path_cost(net.labels, net.open_labels, wl.path)
    path, sliced, info = T.path_optimize(net.labels, net.open_labels, wl.path, seed=5,
                                         sweeps=200, sweeps_final=0, t_start=0.03, t_end=0.001)
    max_log, tcc, _ = W.path_cost(net.labels, net.open_labels, path)
    assert abs(info["initial_log2_tcc"] - math.log2(tcc0)) < 1e-9
    assert abs(info["log2_tcc"] - math.log2(tcc)) < 1e-9
    assert info["max_log2_size"] == max_log
    assert tcc < tcc0 / 4  # annealing from the greedy tree removes most of its work
    alive = set(range(net.num_tensors))
    for a, b in path:  # the pair format of Sec. 3.1: the result keeps id a
        assert a in alive and b in alive
        alive.discard(b)
    assert len(alive) == 1


def test_deterministic_for_a_seed_and_best_of_chains():
    wl = W.small_workload()
    net = wl.network
    kw = dict(sweeps=50, sweeps_final=0, t_start=0.5, t_end=0.01)
    a = T.path_optimize(net.labels, net.open_labels, wl.path, seed=9, **kw)
    b = T.path_optimize(net.labels, net.open_labels, wl.path, seed=9, **kw)
    assert a[0] == b[0] and a[2]["score"] == b[2]["score"]
    c = T.path_optimize(net.labels, net.open_labels, wl.path, seed=9, chains=4, **kw)
    assert c[2]["score"] <= a[2]["score"]  # chain 0 repeats the single chain


def test_dynamic_slicing_meets_the_size_target():
    wl = W.bench_workload()
    net = wl.network
    path, sliced, info = T.path_optimize(net.labels, net.open_labels, wl.path, seed=3,
                                         sweeps=100, sweeps_per_slice=20, sweeps_final=50,
                                         t_start=0.03, t_end=0.001, max_log2_size=24)
    assert info["max_log2_size"] <= 24
    assert info["num_sliced"] == len(sliced) > 0
    assert not set(sliced) & set(net.open_labels)
    assert len(set(sliced)) == len(sliced)
    max_log, tcc, _ = W.path_cost(net.labels, net.open_labels, path, sliced)
    assert max_log <= 24
    assert abs(info["log2_tcc"] - math.log2(tcc)) < 1e-9
    assert abs(info["log2_tcc_total"] - info["log2_tcc"] - len(sliced)) < 1e-12


def test_optimised_path_and_slices_give_the_same_amplitudes():
    # path independence and slice-sum invariance, through the oracle
    wl = W.small_workload()
    net = wl.network
    ref = O.contract(net.tensors, net.labels, net.open_labels, wl.path)
    path, sliced, info = T.path_optimize(net.labels, net.open_labels, wl.path, seed=11,
                                         sweeps=100, sweeps_per_slice=20, sweeps_final=50,
                                         t_start=0.1, t_end=0.001, max_log2_size=7)
    assert info["num_sliced"] >= 1
    got = O.contract(net.tensors, net.labels, net.open_labels, path, sliced)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_argument_checks():
    code = {v: k for k, v in T.STATUS.items()}
    labels, open_labels = [[0, 1], [1, 2], [2, 0]], []
    path = [(0, 1), (0, 2)]
    p, s, info = T.path_optimize(labels, open_labels, path, sweeps=5)
    assert len(p) == 2
    with pytest.raises(T.TnError) as e:  # a retired id reused
        T.path_optimize(labels, open_labels, [(0, 1), (1, 2)])
    assert e.value.status == code["TN_ERR_PATH"]
    with pytest.raises(T.TnError) as e:  # dangling label
        T.path_optimize([[0, 1], [1]], [], [(0, 1)])
    assert e.value.status == code["TN_ERR_SHAPE"]
    with pytest.raises(T.TnError) as e:  # hyperedge
        T.path_optimize([[0, 1], [0, 2], [0, 1, 2]], [], [(0, 1), (0, 2)])
    assert e.value.status == code["TN_ERR_UNSUPPORTED"]
    with pytest.raises(T.TnError) as e:
        T.path_optimize(labels, open_labels, path, t_start=0.01, t_end=0.1)
    assert e.value.status == code["TN_ERR_INVALID_ARG"]


def test_random_greedy_start_beats_the_plain_greedy_tree():
    # 30-qubit bench circuit: random greedy trees (no annealing) against the greedy input path
    wl = W.bench_workload()
    net = wl.network
    _, tcc0, _ = W.path_cost(net.labels, net.open_labels, wl.path)
    path, _, info = T.path_optimize(net.labels, net.open_labels, wl.path, seed=2, sweeps=0,
                                    sweeps_final=0, greedy_trials=20)
    max_log, tcc, _ = W.path_cost(net.labels, net.open_labels, path)
    assert tcc <= tcc0 and abs(info["log2_tcc"] - math.log2(tcc)) < 1e-9
    again, _, _ = T.path_optimize(net.labels, net.open_labels, wl.path, seed=2, sweeps=0,
                                  sweeps_final=0, greedy_trials=20)
    assert again == path
    # the amplitudes along a random greedy tree of the small circuit equal the oracle's
    sw = W.small_workload()
    p2, _, _ = T.path_optimize(sw.network.labels, sw.network.open_labels, sw.path, seed=3,
                               sweeps=0, sweeps_final=0, greedy_trials=10)
    ref = O.contract(sw.network.tensors, sw.network.labels, sw.network.open_labels, sw.path)
    got = O.contract(sw.network.tensors, sw.network.labels, sw.network.open_labels, p2)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_balanced_indices_term():
    # App. A.2: with balance_log2 > 0 the multiply-adds of steps that are unbalanced as GEMMs
    # (k < 64 or min(m, n) < 32) weigh 2^balance_log2 times in the score; the reported T_cc is
    # still the plain count, and the unbalanced share of the work falls
    wl = W.bench_workload()
    net = wl.network

    def unbalanced_share(path):
        steps = W.replay_path(net.labels, net.open_labels, path)
        total = sum(s.tcc for s in steps)
        ub = sum(s.tcc for s in steps
                 if len(s.k_labels) < 6 or min(len(s.m_labels), len(s.n_labels)) < 5)
        return ub / total, total

    kw = dict(seed=5, sweeps=200, sweeps_final=0, t_start=0.03, t_end=0.001, chains=4)
    p0, _, i0 = T.path_optimize(net.labels, net.open_labels, wl.path, **kw)
    p3, _, i3 = T.path_optimize(net.labels, net.open_labels, wl.path, balance_log2=3, **kw)
    f0, t0 = unbalanced_share(p0)
    f3, t3 = unbalanced_share(p3)
    assert abs(i3["log2_tcc"] - math.log2(t3)) < 1e-9 and abs(i0["log2_tcc"] - math.log2(t0)) < 1e-9
    assert f3 < f0 / 4
    again = T.path_optimize(net.labels, net.open_labels, wl.path, balance_log2=0, **kw)
    assert again[0] == p0  # 0 is the default: off
    code = {v: k for k, v in T.STATUS.items()}
    for bad in (-1, 17):
        with pytest.raises(T.TnError) as e:
            T.path_optimize(net.labels, net.open_labels, wl.path, balance_log2=bad, sweeps=1)
        assert e.value.status == code["TN_ERR_INVALID_ARG"]
