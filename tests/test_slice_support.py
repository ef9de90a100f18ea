"""Host-side choice of contributing slices for the 53-qubit parity check (slice_support.py): the
conditions of ``slice_constraints`` are necessary, so every slice whose oracle contraction is
nonzero must meet them, and the seeded search returns only slices that do.  Small Sycamore-shaped
circuits (fSim at theta = pi/2, no final single-qubit layer), sliced to a few bonds; no GPU."""
import numpy as np
import pytest

from paper_2310_03978_gb300 import slice_support as S
from oracle import oracle as O
from paper_2310_03978_gb300 import workload as W


def sliced_circuit(seed, rows, cols, cycles, n_sliced):
    """A seeded circuit with its last two qubits open, the greedy path, and ``n_sliced`` sliced
    bonds: the input wires of last-layer fSims whose outputs are both projected (where slices
    vanish), then greedy choices."""
    circ = W.random_circuit(rows, cols, cycles, seed)
    n = circ.n_qubits
    rng = W.Xoshiro256ss(seed)
    net = W.build_network(circ, [n - 2, n - 1], {q: rng.below(2) for q in range(n - 2)})
    path = W.greedy_path(net.labels, net.open_labels)
    projected = {ls[0] for ls in net.labels[n:] if len(ls) == 1}  # the first n are |0> inputs
    sliced = []
    for ls in net.labels:
        if len(ls) == 4 and ls[0] in projected and ls[1] in projected:
            sliced += [ls[2], ls[3]]
    sliced = sliced[:n_sliced - 1]
    for l in W.greedy_slices(net.labels, net.open_labels, path, n_sliced):
        if len(sliced) < n_sliced and l not in sliced:
            sliced.append(l)
    return net, path, sliced


@pytest.mark.parametrize("seed,shape,n_sliced", [(123, (3, 4, 6), 5), (9, (3, 4, 6), 5),
                                                 (31, (2, 4, 8), 4)])
def test_contributing_slices_meet_the_conditions(seed, shape, n_sliced):
    net, path, sliced = sliced_circuit(seed, *shape, n_sliced)
    cons = S.slice_constraints(net, sliced)
    total = 0.0
    for s in range(1 << len(sliced)):
        a = O.contract(net.tensors, net.labels, net.open_labels, path, sliced, s, s + 1)
        total += np.linalg.norm(a)
        if np.linalg.norm(a) > 1e-12:
            assert S.slice_supported(cons, s), s
    assert total > 0
    # the wires sliced here make most slices vanish, and the conditions see it
    assert sum(S.slice_supported(cons, s) for s in range(1 << len(sliced))) < 1 << len(sliced)
    found = S.supported_slices(net, sliced, 7, 1 << len(sliced))
    assert len(found) == len(set(found))
    assert all(S.slice_supported(cons, s) for s in found)
    assert sorted(found) == [s for s in range(1 << len(sliced)) if S.slice_supported(cons, s)]


def test_a_projector_after_a_swap_like_fsim_fixes_the_partner_wire():
    # two qubits: |0>|0>, sqrtX on both, fSim(pi/2, pi/6), qubit 0 closed on <1|, qubit 1 open;
    # the fSim swaps the wires, so the bond from qubit 1's sqrtX into the fSim must carry 1
    circ = W.Circuit(n_qubits=2)
    circ.gates.append(W.Gate((0,), W.ONE_QUBIT_SET[0], "sqrtX"))
    circ.gates.append(W.Gate((1,), W.ONE_QUBIT_SET[0], "sqrtX"))
    circ.gates.append(W.Gate((0, 1), W.fsim(W.FSIM_THETA, W.FSIM_PHI), "fsim"))
    net = W.build_network(circ, [1], {0: 1})
    fs = net.labels[4]  # (out0, out1, in0, in1)
    in1 = fs[3]
    cons = S.slice_constraints(net, [in1])
    assert not S.slice_supported(cons, 0) and S.slice_supported(cons, 1)
    path = W.greedy_path(net.labels, net.open_labels)
    a0 = O.contract(net.tensors, net.labels, net.open_labels, path, [in1], 0, 1)
    a1 = O.contract(net.tensors, net.labels, net.open_labels, path, [in1], 1, 2)
    assert np.linalg.norm(a0) < 1e-15 and np.linalg.norm(a1) > 0.1
