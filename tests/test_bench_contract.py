"""The reference arm of bench.py (the CPU oracle on the host cores) prints one JSON line with the
benchmark contract's keys; it needs no GPU, so the contract is checked on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["unit"] == "TFLOPS" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "sycamore_5x6_c14_open10_s4"


def test_stored_amplitudes_and_error_measures():
    # bench.py reports its errors against the stored oracle amplitudes with its own measures;
    # both are checked here against the oracle's definitions
    import numpy as np

    import bench
    from oracle import oracle as O
    from paper_2310_03978_gb300 import workload as W
    sizes = {"sycamore_3x4_c8_open6": 64, "sycamore_5x6_c14_open10_s4": 1024,
             "sparse_state_sycamore_4x6_c12_all_open": 4096}
    for name, n in sizes.items():
        g = bench.golden_amps(name)
        assert g is not None and g.shape == (n,) and np.all(np.isfinite(g))
    # the small circuit's stored amplitudes are the state vector's at the open subspace
    wl = W.small_workload()
    net = wl.network
    sv = O.statevector(wl.circuit.n_qubits, wl.circuit.gates)
    idx = [W.full_index(net.n_qubits, net.open_qubits, net.closed_bits, x)
           for x in range(1 << len(net.open_qubits))]
    g = bench.golden_amps("sycamore_3x4_c8_open6")
    assert np.max(np.abs(g - sv[idx])) < 1e-15
    rng = np.random.default_rng(4)
    a = g + 1e-3 * (rng.standard_normal(g.size) + 1j * rng.standard_normal(g.size)) * np.abs(g)
    assert abs(bench.rel_l2(a, g) - O.rel_l2(a, g)) < 1e-15
    assert abs(bench.eps_l2sq(a, g) - O.eps_l2sq(a, g)) < 1e-15
    n = wl.circuit.n_qubits
    assert abs(bench.xeb_ideal(g, n) - O.readout(g, n)[3]) < 1e-9 * abs(O.readout(g, n)[3])
    assert abs(bench.xeb_ideal(a, n) - O.readout(a, n)[3]) < 1e-9 * abs(O.readout(a, n)[3])
