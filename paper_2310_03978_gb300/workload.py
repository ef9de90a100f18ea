"""Seeded synthetic inputs: random circuits, their tensor networks, contraction paths and slices.

This module holds no contraction arithmetic.  It produces the *inputs* of the engine and of the
oracle: gate matrices, the circuit -> tensor-network mapping (paper Sec. 2.1), a greedy pairwise
contraction path (Sec. 3.1 path format: pairs (a, b), the result keeps id a), and a greedy choice
of sliced bonds (Sec. 3.2, dynamic slicing without the re-tuning of the order).

Conventions shared by both sides:
  * qubit q of a rows x cols grid is (r, c) = divmod(q, cols), numbered row-major; removed sites
    are skipped in the numbering;
  * a gate tensor's labels are (outputs..., inputs...); for a 2-qubit gate on (qa, qb) with
    qa < qb the matrix row index is 2*out_a + out_b and the column index 2*in_a + in_b;
  * the amplitude vector's index is built from the open labels in the order given, the first
    open label being the most significant bit; the state vector uses qubit 0 as its MSB.

Random numbers come from xoshiro256** seeded through splitmix64 (Vigna's published generators),
so that the same stream can be re-created in any language.
"""
from __future__ import annotations

import cmath
import heapq
import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
BASE_SEED = 0x231003978


# --------------------------------------------------------------------------------------------
# Random numbers: splitmix64 (seeding) and xoshiro256** (stream), both as published by Vigna.
# --------------------------------------------------------------------------------------------
def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


class Xoshiro256ss:
    def __init__(self, seed: int):
        sm = SplitMix64(seed)
        self.s = [sm.next() for _ in range(4)]

    def next(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = (MASK64 + 1) - ((MASK64 + 1) % n)
        while True:
            x = self.next()
            if x < limit:
                return x % n

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def normal(self) -> float:
        """Standard normal by Box-Muller on two uniforms."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------------------------
# Gate matrices (Sec. 2.2 names the set; the matrices are the standard Sycamore definitions).
# --------------------------------------------------------------------------------------------
_S2 = 1.0 / math.sqrt(2.0)
SQRT_X = np.array([[1, -1j], [-1j, 1]], dtype=np.complex128) * _S2
SQRT_Y = np.array([[1, -1], [1, 1]], dtype=np.complex128) * _S2
SQRT_W = np.array([[1, -cmath.exp(1j * math.pi / 4)], [cmath.exp(-1j * math.pi / 4), 1]],
                  dtype=np.complex128) * _S2
HADAMARD = np.array([[1, 1], [1, -1]], dtype=np.complex128) * _S2
IDENTITY2 = np.eye(2, dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
ONE_QUBIT_SET = (SQRT_X, SQRT_Y, SQRT_W)
ONE_QUBIT_NAMES = ("sqrtX", "sqrtY", "sqrtW")


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, cmath.exp(-1j * phi)]], dtype=np.complex128)


FSIM_THETA = math.pi / 2
FSIM_PHI = math.pi / 6


# --------------------------------------------------------------------------------------------
# Circuits
# --------------------------------------------------------------------------------------------
@dataclass
class Gate:
    qubits: tuple          # (q,) or (qa, qb) with the matrix ordered as documented above
    matrix: np.ndarray     # 2x2 or 4x4 complex128
    name: str = ""


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)
    rows: int = 0
    cols: int = 0


def grid_sites(rows: int, cols: int, removed=()):
    """Row-major qubit numbering of a rows x cols grid with some (r, c) sites removed."""
    removed = set(tuple(x) for x in removed)
    index = {}
    for r in range(rows):
        for c in range(cols):
            if (r, c) not in removed:
                index[(r, c)] = len(index)
    return index


def coupler_patterns(rows: int, cols: int, removed=()):
    """Four matchings A, B, C, D of a rectangular grid.

    A: horizontal (r,c)-(r,c+1) with r+c even; B: horizontal with r+c odd;
    C: vertical (r,c)-(r+1,c) with r+c even;   D: vertical with r+c odd.
    Together they cover every nearest-neighbour coupler exactly once.
    """
    idx = grid_sites(rows, cols, removed)
    pats = {"A": [], "B": [], "C": [], "D": []}
    for r in range(rows):
        for c in range(cols):
            if (r, c) not in idx:
                continue
            if (r, c + 1) in idx:
                pats["A" if (r + c) % 2 == 0 else "B"].append((idx[(r, c)], idx[(r, c + 1)]))
            if (r + 1, c) in idx:
                pats["C" if (r + c) % 2 == 0 else "D"].append((idx[(r, c)], idx[(r + 1, c)]))
    return pats


CYCLE_ORDER = "ABCDCDAB"


def random_circuit(rows: int, cols: int, cycles: int, seed: int, removed=(),
                   theta: float = FSIM_THETA, phi: float = FSIM_PHI, no_repeat: bool = False):
    """Sycamore-shaped random circuit (Sec. 2.2): each cycle is a layer of single-qubit gates
    drawn from {sqrtX, sqrtY, sqrtW} followed by fSim(theta, phi) on one coupler pattern, in
    ABCDCDAB order.  Draws are iid uniform per qubit per cycle unless ``no_repeat``."""
    idx = grid_sites(rows, cols, removed)
    n = len(idx)
    pats = coupler_patterns(rows, cols, removed)
    rng = Xoshiro256ss(seed)
    circ = Circuit(n_qubits=n, rows=rows, cols=cols)
    prev = [-1] * n
    g2 = fsim(theta, phi)
    for t in range(cycles):
        for q in range(n):
            if no_repeat and prev[q] >= 0:
                k = rng.below(2)
                k = k if k < prev[q] else k + 1
            else:
                k = rng.below(3)
            prev[q] = k
            circ.gates.append(Gate((q,), ONE_QUBIT_SET[k], ONE_QUBIT_NAMES[k]))
        for (qa, qb) in pats[CYCLE_ORDER[t % 8]]:
            circ.gates.append(Gate((qa, qb), g2, "fsim"))
    return circ


def hadamard_circuit(n: int) -> Circuit:
    c = Circuit(n_qubits=n)
    for q in range(n):
        c.gates.append(Gate((q,), HADAMARD, "H"))
    return c


def ghz_circuit(n: int) -> Circuit:
    c = Circuit(n_qubits=n)
    c.gates.append(Gate((0,), HADAMARD, "H"))
    for q in range(n - 1):
        c.gates.append(Gate((q, q + 1), CNOT, "cnot"))
    return c


def mirrored_circuit(circ: Circuit) -> Circuit:
    """The circuit followed by its inverse: every gate, then every adjoint in reverse order."""
    out = Circuit(n_qubits=circ.n_qubits, rows=circ.rows, cols=circ.cols)
    out.gates = list(circ.gates)
    for g in reversed(circ.gates):
        out.gates.append(Gate(g.qubits, g.matrix.conj().T.copy(), g.name + "^dag"))
    return out


# --------------------------------------------------------------------------------------------
# Tensor networks (Sec. 2.1)
# --------------------------------------------------------------------------------------------
@dataclass
class Network:
    tensors: list          # list of np.ndarray complex128, shape (2,)*rank
    labels: list           # list of tuples of int labels, one per tensor, row-major order
    open_labels: list      # output order, first = most significant bit
    n_qubits: int = 0
    open_qubits: list = field(default_factory=list)
    closed_bits: dict = field(default_factory=dict)

    @property
    def num_tensors(self) -> int:
        return len(self.tensors)

    def all_labels(self):
        s = set()
        for ls in self.labels:
            s.update(ls)
        return sorted(s)


def build_network(circ: Circuit, open_qubits, closed_bits: dict) -> Network:
    """Map a circuit to a tensor network: |0> vectors on every input wire, one tensor per gate
    (labels: new output wires, then the input wires), and on every closed qubit a projector
    vector <b| on its last wire.  The open qubits' last wires stay open, in the order given."""
    n = circ.n_qubits
    next_label = 0
    wire = []
    tensors, labels = [], []
    for q in range(n):
        wire.append(next_label)
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append((next_label,))
        next_label += 1
    for g in circ.gates:
        k = len(g.qubits)
        outs = []
        for q in g.qubits:
            outs.append(next_label)
            next_label += 1
        ins = [wire[q] for q in g.qubits]
        t = np.asarray(g.matrix, dtype=np.complex128).reshape((2,) * (2 * k))
        tensors.append(t.copy())
        labels.append(tuple(outs) + tuple(ins))
        for q, o in zip(g.qubits, outs):
            wire[q] = o
    open_qubits = list(open_qubits)
    for q in range(n):
        if q in open_qubits:
            continue
        b = int(closed_bits[q])
        v = np.zeros(2, dtype=np.complex128)
        v[b] = 1.0
        tensors.append(v)
        labels.append((wire[q],))
    return Network(tensors=tensors, labels=labels, open_labels=[wire[q] for q in open_qubits],
                   n_qubits=n, open_qubits=open_qubits, closed_bits=dict(closed_bits))


def full_index(n_qubits: int, open_qubits, closed_bits: dict, x: int) -> int:
    """State-vector index (qubit 0 = MSB) of amplitude x of the open subspace."""
    ko = len(open_qubits)
    bits = {}
    for j, q in enumerate(open_qubits):
        bits[q] = (x >> (ko - 1 - j)) & 1
    for q, b in closed_bits.items():
        bits[q] = int(b)
    idx = 0
    for q in range(n_qubits):
        idx = (idx << 1) | bits[q]
    return idx


# --------------------------------------------------------------------------------------------
# Greedy path (Sec. 3.1 format) and greedy slicing (Sec. 3.2)
# --------------------------------------------------------------------------------------------
def _label_counts(labels, open_labels):
    cnt = {}
    for ls in labels:
        for l in ls:
            cnt[l] = cnt.get(l, 0) + 1
    for l in open_labels:
        cnt[l] = cnt.get(l, 0) + 1
    return cnt


def _pair_result(la, lb, cnt):
    """Labels of the pairwise result: every label of A or B that some other tensor (or the
    output) still needs, in A-then-B order; a label seen only by A and B is summed."""
    sa, sb = set(la), set(lb)
    out = []
    for l in la:
        shared = l in sb
        if (not shared) or cnt[l] > 2:
            out.append(l)
    for l in lb:
        if l not in sa:
            out.append(l)
    return tuple(out)


def greedy_path(labels, open_labels, rng: Xoshiro256ss | None = None, temperature: float = 0.0):
    """Greedy pairwise path: repeatedly contract the connected pair that minimises
    size(out) - size(a) - size(b) (sizes in elements, every dim 2); ties go to the smallest
    (a, b).  With a generator and temperature > 0 the choice among the candidates is sampled
    with weights exp(-cost / (T * size scale)) ("random greedy").  Returns pairs (a, b), a < b;
    the result keeps id a."""
    labels = [tuple(x) for x in labels]
    cnt = _label_counts(labels, open_labels)
    alive = {i: labels[i] for i in range(len(labels))}
    owners = {}
    for i, ls in alive.items():
        for l in ls:
            owners.setdefault(l, set()).add(i)
    version = {i: 0 for i in alive}

    def cost(a, b):
        lo = _pair_result(alive[a], alive[b], cnt)
        return (2 ** len(lo)) - (2 ** len(alive[a])) - (2 ** len(alive[b]))

    heap = []

    def push_pairs(i):
        nb = set()
        for l in alive[i]:
            nb.update(owners.get(l, ()))
        nb.discard(i)
        for j in nb:
            a, b = (i, j) if i < j else (j, i)
            heapq.heappush(heap, (cost(a, b), a, b, version[a], version[b]))

    for i in list(alive):
        push_pairs(i)
    path = []
    while len(alive) > 1:
        cand = None
        if rng is not None and temperature > 0.0:
            pool = []
            while heap and len(pool) < 8:
                c, a, b, va, vb = heapq.heappop(heap)
                if a in alive and b in alive and version[a] == va and version[b] == vb:
                    pool.append((c, a, b, va, vb))
            if pool:
                cmin = pool[0][0]
                scale = max(abs(cmin), 1.0)
                ws = [math.exp(-(p[0] - cmin) / (temperature * scale)) for p in pool]
                tot = sum(ws)
                u = rng.uniform() * tot
                pick = len(pool) - 1
                acc = 0.0
                for k, w in enumerate(ws):
                    acc += w
                    if u < acc:
                        pick = k
                        break
                cand = pool[pick]
                for k, p in enumerate(pool):
                    if k != pick:
                        heapq.heappush(heap, p)
        else:
            while heap:
                c, a, b, va, vb = heapq.heappop(heap)
                if a in alive and b in alive and version[a] == va and version[b] == vb:
                    cand = (c, a, b, va, vb)
                    break
        if cand is None:
            ids = sorted(alive)
            a, b = ids[0], ids[1]
        else:
            a, b = cand[1], cand[2]
        lo = _pair_result(alive[a], alive[b], cnt)
        for l in alive[a]:
            owners[l].discard(a)
        for l in alive[b]:
            owners[l].discard(b)
            cnt[l] -= 1 if l in alive[a] else 0
        # a label contracted away leaves the count table; a batch label loses one owner
        for l in set(alive[a]) & set(alive[b]):
            if l not in lo:
                cnt[l] = 0
        del alive[b]
        alive[a] = lo
        version[a] += 1
        for l in lo:
            owners.setdefault(l, set()).add(a)
        path.append((a, b))
        push_pairs(a)
    return path


@dataclass
class StepShape:
    a: int
    b: int
    labels_a: tuple
    labels_b: tuple
    labels_out: tuple
    batch: tuple
    m_labels: tuple
    n_labels: tuple
    k_labels: tuple

    @property
    def log_out(self):
        return len(self.labels_out)

    @property
    def tcc(self):
        """T_cc = 8 * |A| * |B| / |contracted| (Eq. for T_cc, complex multiply-add = 8 flops)."""
        return 8 * (2 ** (len(self.labels_a) + len(self.labels_b) - len(self.k_labels)))


def replay_path(labels, open_labels, path, sliced=()):
    """Shapes of every step of ``path`` after removing the sliced labels."""
    sl = set(sliced)
    cur = {i: tuple(l for l in ls if l not in sl) for i, ls in enumerate(labels)}
    cnt = _label_counts([cur[i] for i in cur], open_labels)
    steps = []
    for (a, b) in path:
        la, lb = cur[a], cur[b]
        lo = _pair_result(la, lb, cnt)
        sa, sb, so = set(la), set(lb), set(lo)
        batch = tuple(l for l in la if l in sb and l in so)
        k = tuple(l for l in la if l in sb and l not in so)
        m = tuple(l for l in la if l not in sb)
        n = tuple(l for l in lb if l not in sa)
        steps.append(StepShape(a, b, la, lb, lo, batch, m, n, k))
        for l in la:
            if l in sb:
                cnt[l] -= 1
        for l in k:
            cnt[l] = 0
        cur[a] = lo
        del cur[b]
    return steps


def path_cost(labels, open_labels, path, sliced=()):
    steps = replay_path(labels, open_labels, path, sliced)
    max_log = max((s.log_out for s in steps), default=0)
    tcc = sum(s.tcc for s in steps)
    return max_log, tcc, steps


def greedy_slices(labels, open_labels, path, num_sliced: int):
    """Greedy slicing: repeatedly cut the bond that most reduces the largest intermediate,
    ties broken by the lower total T_cc and then the lowest label id.  Open labels are never
    sliced."""
    chosen = []
    openset = set(open_labels)
    for _ in range(num_sliced):
        max_log, tcc, steps = path_cost(labels, open_labels, path, chosen)
        cands = set()
        for s in steps:
            if s.log_out == max_log:
                cands.update(s.labels_out)
        cands -= openset
        best = None
        for l in sorted(cands):
            ml, t, _ = path_cost(labels, open_labels, path, chosen + [l])
            key = (ml, t, l)
            if best is None or key < best:
                best = key
        if best is None:
            break
        chosen.append(best[2])
    return chosen


def best_random_greedy(labels, open_labels, seed: int, trials: int, temperature: float):
    """Deterministic greedy first, then ``trials`` random-greedy paths; keeps the path with the
    smallest (largest intermediate, total T_cc)."""
    best_path = greedy_path(labels, open_labels)
    ml, t, _ = path_cost(labels, open_labels, best_path)
    best = (ml, t)
    rng = Xoshiro256ss(seed)
    for _ in range(trials):
        p = greedy_path(labels, open_labels, rng=rng, temperature=temperature)
        ml, t, _ = path_cost(labels, open_labels, p)
        if (ml, t) < best:
            best, best_path = (ml, t), p
    return best_path


# --------------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    circuit: Circuit
    network: Network
    path: list
    sliced: list

    @property
    def num_slices(self) -> int:
        return 1 << len(self.sliced)


def sycamore_workload(name, rows, cols, cycles, k_open, num_sliced, config_id, removed=(),
                      path_trials=0, temperature=0.0):
    """Seeded Sycamore-shaped workload: circuit, network with the last ``k_open`` qubits open and
    the others closed on seeded bits, a (random-)greedy path and ``num_sliced`` greedy slices."""
    seed = BASE_SEED + config_id
    circ = random_circuit(rows, cols, cycles, seed, removed)
    n = circ.n_qubits
    rng = Xoshiro256ss(seed ^ 0x5EED)
    open_q = list(range(n - k_open, n))
    closed = {q: rng.below(2) for q in range(n - k_open)}
    net = build_network(circ, open_q, closed)
    if path_trials > 0:
        path = best_random_greedy(net.labels, net.open_labels, seed ^ 0xFA7, path_trials,
                                  temperature)
    else:
        path = greedy_path(net.labels, net.open_labels)
    sliced = greedy_slices(net.labels, net.open_labels, path, num_sliced) if num_sliced else []
    return Workload(name, circ, net, path, sliced)


def sycamore53_network(cycles=16, k_open=12, config_id=4):
    """The 53-qubit Sycamore-shaped circuit (6x9 grid without site (5, 8)), ``cycles`` cycles,
    the last ``k_open`` qubits open and the others closed on seeded bits.  No path: the greedy
    path is far too costly here; the caller anneals one.  Returns (circuit, network)."""
    seed = BASE_SEED + config_id
    circ = random_circuit(6, 9, cycles, seed, removed=((5, 8),))
    n = circ.n_qubits
    rng = Xoshiro256ss(seed ^ 0x5EED)
    open_q = list(range(n - k_open, n))
    closed = {q: rng.below(2) for q in range(n - k_open)}
    return circ, build_network(circ, open_q, closed)


def sycamore45_network(cycles=14, k_open=12, config_id=6):
    """A 45-qubit Sycamore-shaped circuit (5x9 grid), ``cycles`` cycles, the last ``k_open``
    qubits open and the others closed on seeded bits: the shape of the paper's 45-qubit 14-cycle
    precision study (Sec. 4.3, Tables 2-3).  No path: the caller anneals one.  Returns (circuit,
    network)."""
    seed = BASE_SEED + config_id
    circ = random_circuit(5, 9, cycles, seed)
    n = circ.n_qubits
    rng = Xoshiro256ss(seed ^ 0x5EED)
    open_q = list(range(n - k_open, n))
    closed = {q: rng.below(2) for q in range(n - k_open)}
    return circ, build_network(circ, open_q, closed)


def sparse_state_workload(rows=4, cols=6, cycles=12, num_samples=4096, config_id=9):
    """Sparse-state input (Sec. 3.3): a seeded Sycamore-shaped circuit with every qubit open and
    ``num_samples`` seeded uniform bitstrings standing in for sampled ones (column j = qubit j,
    the network's open label j).  Returns (circuit, network, samples as an (S, n) uint8 array)."""
    seed = BASE_SEED + config_id
    circ = random_circuit(rows, cols, cycles, seed)
    n = circ.n_qubits
    net = build_network(circ, list(range(n)), {})
    rng = Xoshiro256ss(seed ^ 0x5A4D)
    smp = np.zeros((num_samples, n), dtype=np.uint8)
    for i in range(num_samples):
        x = rng.next()
        for j in range(n):
            smp[i, j] = (x >> j) & 1
    return circ, net, smp


def small_workload() -> Workload:
    """12-qubit 3x4 grid, 8 cycles, 6 open qubits (64 amplitudes), greedy path, no slicing."""
    return sycamore_workload("sycamore_3x4_c8_open6", 3, 4, 8, 6, 0, 0)


def bench_workload() -> Workload:
    """30-qubit 5x6 grid, 14 cycles, 10 open qubits (1024 amplitudes), 4 sliced bonds (16
    slices); best of one greedy and 20 random-greedy paths (T = 0.05); the largest sliced
    intermediate is 2^28 elements."""
    return sycamore_workload("sycamore_5x6_c14_open10_s4", 5, 6, 14, 10, 4, 1,
                             path_trials=20, temperature=0.05)
