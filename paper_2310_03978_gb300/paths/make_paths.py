"""Write the stored contraction paths of the large Sycamore-shaped circuits.

The bench contracts the 53-qubit 16- and 20-cycle circuits (6x9 grid without site (5, 8)) and
the 45-qubit 14-cycle circuit (5x9 grid), each with 12 open qubits, along paths from the
annealing optimiser (tn_path_optimize: random greedy initial
trees, simulated annealing with the paper's local three-descendant update, then dynamic slicing
with re-tuning sweeps after each sliced bond, Sec. 3.2).  Finding them takes minutes of host
time, so they are computed once by this script and stored as JSON beside it:

    python -m paper_2310_03978_gb300.paths.make_paths [16] [20] [sycamore45_5x9_c14_open12]

Each file holds the path (pairs, the result keeps the first id), the sliced labels (bit j of a
slice id is the value of sliced[j]), the optimiser's settings and its cost figures.  The
network itself is rebuilt from its seed (``network``).
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEED = 7
# name: (builder arguments, size cap log2, sweeps before slicing, re-tuning sweeps per bond)
SETTINGS = {
    "sycamore53_6x9_c16_open12": (("sycamore53", 16, 4), 30, 8000, 300),
    "sycamore53_6x9_c20_open12": (("sycamore53", 20, 5), 31, 8000, 300),
    "sycamore45_5x9_c14_open12": (("sycamore45", 14, 6), 26, 2000, 60),
}


def name_of(cycles_or_name) -> str:
    if isinstance(cycles_or_name, str):
        return cycles_or_name
    return "sycamore53_6x9_c%d_open12" % cycles_or_name


def network(name: str):
    """(circuit, network) of a named workload, rebuilt from its seed."""
    from paper_2310_03978_gb300 import workload as W
    (kind, cycles, config_id), _, _, _ = SETTINGS[name]
    if kind == "sycamore53":
        return W.sycamore53_network(cycles=cycles, config_id=config_id)
    return W.sycamore45_network(cycles=cycles, config_id=config_id)


def path_file(cycles_or_name) -> str:
    return os.path.join(HERE, name_of(cycles_or_name) + ".json")


def make(name: str) -> dict:
    from paper_2310_03978_gb300 import tn, workload as W
    (kind, cycles, config_id), cap, sweeps, retune = SETTINGS[name]
    _, net = network(name)
    t0 = time.perf_counter()
    g = W.greedy_path(net.labels, net.open_labels)
    path, _, _ = tn.path_optimize(net.labels, net.open_labels, g, seed=SEED, sweeps=sweeps,
                                  sweeps_final=0, t_start=0.01, t_end=0.0005, chains=16,
                                  greedy_trials=100, beta=1.0)
    path, sliced, info = tn.path_optimize(net.labels, net.open_labels, path, seed=SEED + 1,
                                          sweeps=0, sweeps_per_slice=retune, sweeps_final=300,
                                          t_start=0.005, t_end=0.0005, chains=16,
                                          max_log2_size=cap)
    secs = time.perf_counter() - t0
    return {"workload": name, "cycles": cycles,
            "config_id": config_id, "max_log2_size_cap": cap,
            "optimiser": "tn_path_optimize: greedy start, 100 random greedy trees x 16 chains, "
                         "%d sweeps (T 0.01 -> 0.0005, beta 1), seed %d; then dynamic slicing "
                         "to 2^%d with %d re-tuning sweeps per bond and 300 final sweeps "
                         "(T 0.005 -> 0.0005), seed %d" % (sweeps, SEED, cap, retune, SEED + 1),
            "optimiser_s": secs, "num_sliced": len(sliced),
            "log2_flops_per_slice": info["log2_tcc"],
            "log2_flops_total": info["log2_tcc_total"],
            "max_log2_size": info["max_log2_size"],
            "path": [list(p) for p in path], "sliced": list(sliced)}


def load(cycles_or_name):
    """The stored record (dict) of a named workload's path (53-qubit ones also by cycle count),
    or None when it has not been written."""
    f = path_file(cycles_or_name)
    if not os.path.exists(f):
        return None
    with open(f) as fh:
        return json.load(fh)


if __name__ == "__main__":
    for name in sys.argv[1:] or list(SETTINGS):
        rec = make(name_of(int(name)) if name.isdigit() else name)
        with open(path_file(rec["workload"]), "w") as fh:
            json.dump(rec, fh)
        print(rec["workload"], ":", rec["num_sliced"], "sliced bonds, 2^%.2f flops per slice, "
              "2^%.2f in total, %.0f s" % (rec["log2_flops_per_slice"], rec["log2_flops_total"],
                                           rec["optimiser_s"]))
