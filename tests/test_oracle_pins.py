"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* library special cases of the pairwise einsum (Sec. 2.4): matmul, outer product, tensordot,
  batched matmul, transpose, and numpy's einsum on random all-dim-2 tensors;
* closed forms of the circuit model (Sec. 2.1): all-Hadamard, GHZ, mirrored circuits, explicit
  Kronecker products for 1- and 2-qubit gates;
* brute force: the tensor-network contraction equals the state vector (<= 12 qubits);
* invariants: unit norm, slice sum = unsliced (Sec. 3.2), path independence (Sec. 3.1);
* readout (Eq. lxeb_2) on hand-computed cases.
Mutation tests at the end plant plausible mistakes and check that a pin catches them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_03978_gb300 import workload as W


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- einsum special cases
def test_einsum_matmul():
    rng = np.random.default_rng(1)
    A, B = crandn(rng, 3, 4), crandn(rng, 4, 5)
    C = O.einsum_pair(A, [0, 1], B, [1, 2], [0, 2])
    np.testing.assert_allclose(C, A @ B, rtol=1e-13, atol=1e-13)


def test_einsum_output_transposed():
    rng = np.random.default_rng(2)
    A, B = crandn(rng, 3, 4), crandn(rng, 4, 5)
    C = O.einsum_pair(A, [0, 1], B, [1, 2], [2, 0])
    np.testing.assert_allclose(C, (A @ B).T, rtol=1e-13, atol=1e-13)


def test_einsum_outer_and_scalar():
    rng = np.random.default_rng(3)
    a, b = crandn(rng, 4), crandn(rng, 3)
    np.testing.assert_allclose(O.einsum_pair(a, [0], b, [1], [0, 1]), np.outer(a, b), rtol=1e-13)
    s = O.einsum_pair(a, [0], a.conj(), [0], [])
    assert abs(complex(s.reshape(())) - np.vdot(a, a)) < 1e-12


def test_einsum_tensordot_two_labels():
    rng = np.random.default_rng(4)
    A, B = crandn(rng, 2, 3, 4), crandn(rng, 3, 4, 5)
    C = O.einsum_pair(A, [0, 1, 2], B, [1, 2, 3], [0, 3])
    np.testing.assert_allclose(C, np.tensordot(A, B, axes=([1, 2], [0, 1])), rtol=1e-12)


def test_einsum_batch_label():
    rng = np.random.default_rng(5)
    A, B = crandn(rng, 3, 2, 4), crandn(rng, 3, 4, 2)
    C = O.einsum_pair(A, [9, 0, 1], B, [9, 1, 2], [9, 0, 2])
    np.testing.assert_allclose(C, np.matmul(A, B), rtol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_einsum_random_bit_tensors_vs_numpy(seed):
    rng = np.random.default_rng(100 + seed)
    labels = list(range(12))
    rng.shuffle(labels)
    ra, rb = int(rng.integers(3, 8)), int(rng.integers(2, 7))
    la = [int(x) for x in labels[:ra]]
    lb = [int(x) for x in rng.permutation(labels[max(0, ra - 3):ra + rb])][:rb]
    shared = [l for l in la if l in lb]
    keep = [l for l in la if l not in shared] + [l for l in lb if l not in la]
    keep = [int(x) for x in rng.permutation(keep)]
    if shared and rng.integers(2):
        keep.append(shared[0])  # a batch label
    A, B = crandn(rng, *([2] * ra)), crandn(rng, *([2] * rb))
    letters = "abcdefghijklmnop"
    spec = "%s,%s->%s" % ("".join(letters[l] for l in la), "".join(letters[l] for l in lb),
                          "".join(letters[l] for l in keep))
    C = O.einsum_pair(A, la, B, lb, keep)
    np.testing.assert_allclose(C, np.einsum(spec, A, B), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- gates and the state vector
def test_gate_matrices():
    for g in W.ONE_QUBIT_SET + (W.fsim(W.FSIM_THETA, W.FSIM_PHI),):
        n = g.shape[0]
        np.testing.assert_allclose(g @ g.conj().T, np.eye(n), atol=1e-15)
    X = np.array([[0, 1], [1, 0]])
    np.testing.assert_allclose(W.SQRT_X @ W.SQRT_X, -1j * X, atol=1e-15)
    Y = np.array([[0, -1j], [1j, 0]])
    np.testing.assert_allclose(W.SQRT_Y @ W.SQRT_Y, -1j * Y, atol=1e-15)
    Wm = (X + Y) / math.sqrt(2)
    np.testing.assert_allclose(W.SQRT_W @ W.SQRT_W, -1j * Wm, atol=1e-15)
    # fSim(theta, phi)^dagger = fSim(-theta, -phi)
    np.testing.assert_allclose(W.fsim(0.3, 0.7).conj().T, W.fsim(-0.3, -0.7), atol=1e-15)


def test_statevector_kron_one_and_two_qubit():
    rng = np.random.default_rng(7)
    G = np.linalg.qr(crandn(rng, 2, 2))[0]
    M = np.linalg.qr(crandn(rng, 4, 4))[0]
    e0 = np.zeros(8, dtype=complex)
    e0[0] = 1
    I2 = np.eye(2)
    # qubit 0 is the most significant bit
    sv = O.statevector(3, [W.Gate((0,), G)])
    np.testing.assert_allclose(sv, np.kron(G, np.kron(I2, I2)) @ e0, atol=1e-14)
    sv = O.statevector(3, [W.Gate((2,), G)])
    np.testing.assert_allclose(sv, np.kron(np.kron(I2, I2), G) @ e0, atol=1e-14)
    # a 2-qubit gate on (0, 1), after a layer that populates every basis state
    pre = [W.Gate((q,), W.HADAMARD) for q in range(3)]
    psi = np.kron(W.HADAMARD, np.kron(W.HADAMARD, W.HADAMARD)) @ e0
    sv = O.statevector(3, pre + [W.Gate((0, 1), M)])
    np.testing.assert_allclose(sv, np.kron(M, I2) @ psi, atol=1e-14)
    # reversed qubit order (1, 0): the swap-conjugated matrix
    SW = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]])
    sv = O.statevector(3, pre + [W.Gate((1, 0), M)])
    np.testing.assert_allclose(sv, np.kron(SW @ M @ SW, I2) @ psi, atol=1e-14)


def test_statevector_closed_forms():
    n = 6
    sv = O.statevector(n, W.hadamard_circuit(n).gates)
    np.testing.assert_allclose(sv, np.full(1 << n, 2 ** (-n / 2)), atol=1e-14)
    sv = O.statevector(n, W.ghz_circuit(n).gates)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(sv, ref, atol=1e-14)
    circ = W.random_circuit(2, 3, 5, seed=11)
    sv = O.statevector(circ.n_qubits, W.mirrored_circuit(circ).gates)
    ref = np.zeros(1 << circ.n_qubits, dtype=complex)
    ref[0] = 1
    np.testing.assert_allclose(sv, ref, atol=1e-13)
    sv = O.statevector(circ.n_qubits, circ.gates)
    assert abs(np.sum(np.abs(sv) ** 2) - 1) < 1e-13


# ---------------------------------------------------------------- contraction vs brute force
def _network_all_open(circ):
    return W.build_network(circ, list(range(circ.n_qubits)), {})


def test_contract_hadamard_and_ghz_closed_forms():
    n = 7
    net = _network_all_open(W.hadamard_circuit(n))
    path = W.greedy_path(net.labels, net.open_labels)
    amps = O.contract_network(net, path)
    np.testing.assert_allclose(amps, np.full(1 << n, 2 ** (-n / 2)), atol=1e-14)
    net = _network_all_open(W.ghz_circuit(n))
    amps = O.contract_network(net, W.greedy_path(net.labels, net.open_labels))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(amps, ref, atol=1e-14)


def test_contract_mirrored_circuit_is_identity():
    circ = W.mirrored_circuit(W.random_circuit(2, 3, 4, seed=5))
    net = _network_all_open(circ)
    amps = O.contract_network(net, W.greedy_path(net.labels, net.open_labels))
    ref = np.zeros(1 << circ.n_qubits, dtype=complex)
    ref[0] = 1
    np.testing.assert_allclose(amps, ref, atol=1e-13)


def test_contract_all_open_matches_statevector_and_norm():
    circ = W.random_circuit(3, 3, 6, seed=21)
    net = _network_all_open(circ)
    amps = O.contract_network(net, W.greedy_path(net.labels, net.open_labels))
    sv = O.statevector(circ.n_qubits, circ.gates)
    np.testing.assert_allclose(amps, sv, atol=1e-13)
    assert abs(np.sum(np.abs(amps) ** 2) - 1) < 1e-12


def test_contract_small_workload_matches_statevector():
    wl = W.small_workload()
    amps = O.contract_network(wl.network, wl.path)
    sv = O.statevector(wl.circuit.n_qubits, wl.circuit.gates)
    net = wl.network
    idx = [W.full_index(net.n_qubits, net.open_qubits, net.closed_bits, x)
           for x in range(1 << len(net.open_qubits))]
    np.testing.assert_allclose(amps, sv[idx], rtol=0, atol=1e-13)
    assert O.rel_l2(amps, sv[idx]) < 1e-12


def test_slice_sum_equals_unsliced_and_ranges_split():
    wl = W.small_workload()
    net = wl.network
    full = O.contract_network(net, wl.path)
    sliced = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    assert len(sliced) == 3
    s_all = O.contract_network(net, wl.path, sliced)
    np.testing.assert_allclose(s_all, full, atol=1e-13)
    a = O.contract_network(net, wl.path, sliced, 0, 3)
    b = O.contract_network(net, wl.path, sliced, 3, 8)
    np.testing.assert_allclose(a + b, full, atol=1e-13)
    # a single slice is not the whole answer
    assert O.rel_l2(a, full) > 1e-3


def test_path_independence():
    wl = W.small_workload()
    net = wl.network
    p1 = wl.path
    p2 = W.greedy_path(net.labels, net.open_labels, rng=W.Xoshiro256ss(99), temperature=1.0)
    assert p1 != p2
    np.testing.assert_allclose(O.contract_network(net, p1), O.contract_network(net, p2),
                               atol=1e-13)


# ---------------------------------------------------------------- readout (Eq. lxeb_2)
def test_readout_hand_cases():
    out = O.readout(np.array([1, 0, 0, 0], dtype=complex), 2)
    np.testing.assert_allclose(out, [1.0, 1.0, 4 * 1 / 4 - 1, 4 * 1 / 1 - 1])
    n = 5
    amps = np.full(8, 2 ** (-n / 2), dtype=complex)
    out = O.readout(amps, n)
    np.testing.assert_allclose(out[:2], [8 * 2.0 ** -n, 8 * 2.0 ** (-2 * n)], rtol=1e-15)
    assert abs(out[2] - (2 ** n * 8 * 2.0 ** -n / 8 - 1)) < 1e-15  # = 0
    assert abs(out[3]) < 1e-14


def test_readout_porter_thomas_random_circuit():
    circ = W.random_circuit(3, 4, 12, seed=3)
    sv = O.statevector(circ.n_qubits, circ.gates)
    out = O.readout(sv, circ.n_qubits)
    assert abs(out[0] - 1) < 1e-12
    # every amplitude of the full space is a sample of the ideal distribution: F_l = 0
    assert abs(out[2]) < 1e-12
    # Porter-Thomas: D * E[p^2] / E[p] = 2, so the ideal-sample XEB is near 1
    assert 0.7 < out[3] < 1.3


def test_error_metrics():
    ref = np.array([1.0, 1.0j, 0.0])
    a = np.array([1.0, 1.0j, 0.1])
    assert abs(O.rel_l2(a, ref) - 0.1 / math.sqrt(2)) < 1e-15
    assert abs(O.eps_l2sq(a, ref) - 0.01 / 2) < 1e-15
    assert abs(O.eps_f(1e-4, 0.5) - 1e-4 * 1.5 / 0.5) < 1e-18


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_transposed_operand():
    rng = np.random.default_rng(8)
    A, B = crandn(rng, 4, 4), crandn(rng, 4, 4)
    wrong = O.einsum_pair(A, [1, 0], B, [1, 2], [0, 2])  # A used transposed
    assert np.abs(wrong - A @ B).max() > 1e-3


def test_pins_catch_wrong_qubit_order():
    rng = np.random.default_rng(9)
    G = np.linalg.qr(crandn(rng, 2, 2))[0]
    e0 = np.zeros(4, dtype=complex)
    e0[0] = 1
    sv = O.statevector(2, [W.Gate((1,), G)])
    assert np.abs(sv - np.kron(G, np.eye(2)) @ e0).max() > 1e-3


# ---------------------------------------------------------------- sparse-state contraction
def _samples(rng, n_rows, n_bits, dup=True):
    s = rng.integers(0, 2, size=(n_rows, n_bits))
    if dup:  # repeated bitstrings must give repeated amplitudes
        s[1] = s[0]
        s[-1] = s[2]
    return s


def _sv_index(bits):
    # qubit 0 = most significant bit of the state-vector index
    return int("".join(str(int(b)) for b in bits), 2)


def test_sparse_state_matches_the_state_vector_at_the_samples():
    circ = W.random_circuit(3, 4, 8, seed=31)
    net = _network_all_open(circ)
    path = W.greedy_path(net.labels, net.open_labels)
    rng = np.random.default_rng(5)
    smp = _samples(rng, 48, circ.n_qubits)
    got = O.contract_sparse(net.tensors, net.labels, net.open_labels, path, smp)
    sv = O.statevector(circ.n_qubits, circ.gates)
    np.testing.assert_allclose(got, sv[[_sv_index(r) for r in smp]], rtol=0, atol=1e-13)


def test_sparse_state_closed_forms():
    n = 6
    net = _network_all_open(W.ghz_circuit(n))
    path = W.greedy_path(net.labels, net.open_labels)
    smp = np.array([[0] * n, [1] * n, [1] + [0] * (n - 1), [0, 1] * (n // 2)])
    got = O.contract_sparse(net.tensors, net.labels, net.open_labels, path, smp)
    np.testing.assert_allclose(got, [2 ** -0.5, 2 ** -0.5, 0, 0], atol=1e-14)
    net = _network_all_open(W.hadamard_circuit(n))
    smp = np.random.default_rng(2).integers(0, 2, size=(10, n))
    got = O.contract_sparse(net.tensors, net.labels, net.open_labels,
                            W.greedy_path(net.labels, net.open_labels), smp)
    np.testing.assert_allclose(got, np.full(10, 2 ** (-n / 2)), atol=1e-14)


def test_sparse_state_with_closed_qubits_and_any_path():
    # a batch of open qubits among closed ones; the dense contraction over all open bitstrings,
    # read at the samples, and two different paths agree
    wl = W.small_workload()
    net = wl.network
    rng = np.random.default_rng(13)
    smp = _samples(rng, 20, len(net.open_labels))
    dense = O.contract_network(net, wl.path)
    idx = [_sv_index(r) for r in smp]
    got = O.contract_sparse(net.tensors, net.labels, net.open_labels, wl.path, smp)
    np.testing.assert_allclose(got, dense[idx], rtol=0, atol=1e-13)
    other = W.greedy_path(net.labels, net.open_labels, rng=W.Xoshiro256ss(4), temperature=1.0)
    got2 = O.contract_sparse(net.tensors, net.labels, net.open_labels, other, smp)
    np.testing.assert_allclose(got2, dense[idx], rtol=0, atol=1e-13)


def test_pins_catch_a_swapped_sample_column():
    circ = W.random_circuit(2, 3, 6, seed=7)
    net = _network_all_open(circ)
    path = W.greedy_path(net.labels, net.open_labels)
    smp = np.random.default_rng(3).integers(0, 2, size=(16, circ.n_qubits))
    sv = O.statevector(circ.n_qubits, circ.gates)
    wrong = O.contract_sparse(net.tensors, net.labels, net.open_labels, path, smp[:, ::-1])
    assert np.abs(wrong - sv[[_sv_index(r) for r in smp]]).max() > 1e-3
