"""Write the stored expected amplitudes of the named workloads.

Every value here comes from the CPU oracle: its state-vector simulator (oracle.statevector, a
brute-force application of every gate matrix to the full 2^n state), read at the workload's open
subspace (or, for the sparse-state workload, at its sampled bitstrings), or, for the 45-qubit
circuit (too large for a state vector), its pairwise contraction of a few slices.  Nothing here touches
the GPU path.  bench.py reads these files for the errors it reports.

    python tests/golden/make_golden.py [small|bench|sparse|table3 ...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2310_03978_gb300 import workload as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, wl):
    t0 = time.time()
    net = wl.network
    sv = O.statevector(wl.circuit.n_qubits, wl.circuit.gates)
    idx = [W.full_index(net.n_qubits, net.open_qubits, net.closed_bits, x)
           for x in range(1 << len(net.open_qubits))]
    amps = sv[idx]
    norm = float(np.sum(np.abs(sv) ** 2))
    del sv
    path = os.path.join(HERE, name + ".amps.txt")
    with open(path, "w") as f:
        f.write("# %s: %d qubits, open qubits %s, closed bits seeded; amplitudes from the\n"
                % (wl.name, net.n_qubits, net.open_qubits))
        f.write("# oracle state vector (qubit 0 = MSB), index = open bits, first open qubit = MSB\n")
        f.write("# full-state norm %.17g, oracle threads %d, %.1f s\n"
                % (norm, O.num_threads(), time.time() - t0))
        for a in amps:
            f.write("%.17e %.17e\n" % (a.real, a.imag))
    print("wrote", path, "in %.1f s" % (time.time() - t0))


def write_sparse(name):
    """The 24-qubit all-open circuit of the sparse-state workload: the state-vector amplitude of
    each of its 4096 seeded bitstrings (row i = sample i, qubit 0 = MSB of the index)."""
    t0 = time.time()
    circ, _, smp = W.sparse_state_workload()
    sv = O.statevector(circ.n_qubits, circ.gates)
    amps = sv[[int("".join(str(int(b)) for b in r), 2) for r in smp]]
    norm = float(np.sum(np.abs(sv) ** 2))
    del sv
    path = os.path.join(HERE, name + ".amps.txt")
    with open(path, "w") as f:
        f.write("# %s: %d qubits, all open; amplitude of each of the %d seeded samples from the\n"
                % (name, circ.n_qubits, len(smp)))
        f.write("# oracle state vector (qubit 0 = MSB), one row per sample\n")
        f.write("# full-state norm %.17g, oracle threads %d, %.1f s\n"
                % (norm, O.num_threads(), time.time() - t0))
        for a in amps:
            f.write("%.17e %.17e\n" % (a.real, a.imag))
    print("wrote", path, "in %.1f s" % (time.time() - t0))


def write_slices(name, count):
    """A large stored-path workload (paths/make_paths.py): the oracle's complex128 contraction of
    ``count`` contributing slices (slice ids from slice_support.supported_slices, seed 7; slices
    whose contraction is exactly zero are skipped), summed in increasing slice order.  The slice
    ids are listed in the header."""
    from paper_2310_03978_gb300 import slice_support as S
    from paper_2310_03978_gb300.paths import make_paths as MP
    t0 = time.time()
    rec = MP.load(name)
    _, net = MP.network(name)
    path = [tuple(p) for p in rec["path"]]
    sliced = rec["sliced"]
    found = {}
    for s in S.supported_slices(net, sliced, 7, 3 * count):
        if len(found) == count:
            break
        r = O.contract_network(net, path, sliced, s, s + 1)
        if np.linalg.norm(r) > 0:
            found[s] = r
        print("slice", s, "norm %.3e" % np.linalg.norm(r), "%.0f s" % (time.time() - t0),
              flush=True)
    order = sorted(found)
    amps = found[order[0]].copy()
    for s in order[1:]:  # summed in increasing slice order
        amps = amps + found[s]
    path_out = os.path.join(HERE, name + ".slices.amps.txt")
    with open(path_out, "w") as f:
        f.write("# %s: sum of the oracle's complex128 contractions of slices %s along the stored\n"
                % (name, " ".join(str(s) for s in order)))
        f.write("# path (%d sliced bonds); index = open bits, first open qubit = MSB\n"
                % len(sliced))
        f.write("# slices: %s\n" % " ".join(str(s) for s in order))
        f.write("# oracle threads %d, %.1f s\n" % (O.num_threads(), time.time() - t0))
        for a in amps:
            f.write("%.17e %.17e\n" % (a.real, a.imag))
    print("wrote", path_out, "in %.1f s" % (time.time() - t0))


if __name__ == "__main__":
    which = sys.argv[1:] or ["small", "bench", "sparse"]
    if "table3" in which:
        write_slices("sycamore45_5x9_c14_open12", 4)
    if "small" in which:
        write("sycamore_3x4_c8_open6", W.small_workload())
        # the same circuit with every qubit open (the amplitude-batch measurement)
        wl = W.small_workload()
        n = wl.circuit.n_qubits
        net = W.build_network(wl.circuit, list(range(n)), {})
        write("sycamore_3x4_c8_all_open", W.Workload("sycamore_3x4_c8_all_open", wl.circuit, net,
                                                     [], []))
    if "bench" in which:
        write("sycamore_5x6_c14_open10_s4", W.bench_workload())
    if "sparse" in which:
        write_sparse("sparse_state_sycamore_4x6_c12_all_open")
