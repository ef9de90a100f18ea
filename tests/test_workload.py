"""Seeded input generators: published RNG test vectors, grid couplers, network structure, path
format (Sec. 3.1: pairs, the result keeps the first id) and greedy slicing."""
import numpy as np

from paper_2310_03978_gb300 import workload as W


def test_splitmix64_published_vector():
    s = W.SplitMix64(1234567)
    assert [s.next() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                            9817491932198370423]


def test_xoshiro256ss_published_vector():
    x = W.Xoshiro256ss(0)
    x.s = [1, 2, 3, 4]
    assert [x.next() for _ in range(4)] == [11520, 0, 1509978240, 1215971899390074240]


def test_coupler_patterns_cover_grid_once():
    for rows, cols, removed in [(3, 4, ()), (5, 6, ()), (6, 9, ((5, 8),))]:
        pats = W.coupler_patterns(rows, cols, removed)
        edges = [e for p in "ABCD" for e in pats[p]]
        assert len(edges) == len(set(edges))
        idx = W.grid_sites(rows, cols, removed)
        expect = 0
        for (r, c) in idx:
            expect += ((r, c + 1) in idx) + ((r + 1, c) in idx)
        assert len(edges) == expect
        for p in "ABCD":  # each pattern is a matching
            qs = [q for e in pats[p] for q in e]
            assert len(qs) == len(set(qs))
    assert len(W.grid_sites(6, 9, ((5, 8),))) == 53


def test_network_structure_and_path_format():
    wl = W.small_workload()
    net = wl.network
    cnt = {}
    for ls in net.labels:
        for l in ls:
            cnt[l] = cnt.get(l, 0) + 1
    for l, c in cnt.items():
        assert c == 2 or (c == 1 and l in net.open_labels)
    assert len(wl.path) == net.num_tensors - 1
    alive = set(range(net.num_tensors))
    for a, b in wl.path:
        assert a in alive and b in alive and a < b
        alive.discard(b)
    assert alive == {0} or len(alive) == 1


def test_bench_workload_shape():
    wl = W.bench_workload()
    assert wl.circuit.n_qubits == 30 and len(wl.network.open_labels) == 10
    assert len(wl.sliced) == 4 and not set(wl.sliced) & set(wl.network.open_labels)
    max_log, tcc, steps = W.path_cost(wl.network.labels, wl.network.open_labels, wl.path,
                                      wl.sliced)
    assert max_log <= 28
    assert tcc == sum(s.tcc for s in steps)


def test_circuit_is_seeded():
    a = W.random_circuit(3, 4, 8, 5)
    b = W.random_circuit(3, 4, 8, 5)
    c = W.random_circuit(3, 4, 8, 6)
    assert [g.name for g in a.gates] == [g.name for g in b.gates]
    assert [g.name for g in a.gates] != [g.name for g in c.gates]
