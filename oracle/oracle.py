"""Python access to the CPU oracle (``tn_oracle.c``) — TEST INFRASTRUCTURE ONLY.

The oracle is a plain complex128 C implementation of the method's definitions (pairwise einsum
of Sec. 2.4, path and slicing of Sec. 3.1-3.2, readout of Eq. lxeb_2) plus an independent
state-vector simulator.  Only the tests, the smoke check and the benchmark's CPU-baseline leg use
it; the GPU library neither links nor calls it.

Error metrics written out from the paper:
  * ``rel_l2``        ||a - a_ref||_2 / ||a_ref||_2
  * ``eps_l2sq``      |L2^2 - L2'^2| / L2^2                       (Eq. l2_squared_error)
  * ``eps_f``         eps_l2sq * (1 + F) / F                      (Eq. lxeb_as_l2_error)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tn_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libtn_oracle.so")
_lock = threading.Lock()
_lib = None

_c = ctypes
_cplx_p = _c.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the shared-library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_einsum_pair.restype = _c.c_int
            L.orc_einsum_pair.argtypes = [_c.c_int, _c.c_void_p, _c.c_void_p,
                                          _c.c_int, _c.c_void_p, _c.c_void_p,
                                          _c.c_int, _c.c_void_p, _c.c_void_p, _c.c_void_p]
            L.orc_contract.restype = _c.c_int
            L.orc_contract.argtypes = [_c.c_int, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                                       _c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p,
                                       _c.c_int, _c.c_void_p, _c.c_int, _c.c_void_p,
                                       _c.c_int64, _c.c_int64, _c.c_void_p]
            L.orc_statevector.restype = _c.c_int
            L.orc_statevector.argtypes = [_c.c_int, _c.c_int, _c.c_void_p, _c.c_void_p,
                                          _c.c_void_p, _c.c_void_p]
            L.orc_readout.restype = _c.c_int
            L.orc_readout.argtypes = [_c.c_int64, _c.c_void_p, _c.c_int, _c.c_void_p]
            L.orc_num_threads.restype = _c.c_int
            L.orc_num_threads.argtypes = []
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def einsum_pair(A, labels_a, B, labels_b, labels_c, label_dim=None):
    """C[labels_c] = sum over the other labels of A[labels_a] * B[labels_b] (Eq. chap2_einsum)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    la, lb, lc = _i32(labels_a), _i32(labels_b), _i32(labels_c)
    if label_dim is None:
        nl = 1 + max([0] + list(la) + list(lb) + list(lc))
        dims = np.zeros(nl, dtype=np.int32)
        for l, d in zip(la, A.shape):
            dims[l] = d
        for l, d in zip(lb, B.shape):
            dims[l] = d
    else:
        dims = _i32(label_dim)
    shape_c = tuple(int(dims[l]) for l in lc)
    C = np.zeros(shape_c, dtype=np.complex128)
    rc = lib().orc_einsum_pair(len(la), la.ctypes.data, A.ctypes.data, len(lb), lb.ctypes.data,
                               B.ctypes.data, len(lc), lc.ctypes.data, C.ctypes.data,
                               dims.ctypes.data)
    if rc != 0:
        raise ValueError("orc_einsum_pair failed: %d" % rc)
    return C


def contract(tensors, labels, open_labels, path, sliced=(), slice_begin=0, slice_end=None,
             label_dim=None):
    """Sum over slices [slice_begin, slice_end) of the contraction along ``path`` (Sec. 3.1-3.2).
    Returns the amplitude vector indexed by ``open_labels`` (first = most significant)."""
    n = len(tensors)
    ts = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
    ls = [_i32(l) for l in labels]
    nl = 1 + max([0] + [int(x) for l in ls for x in l] + list(open_labels))
    if label_dim is None:
        dims = np.zeros(nl, dtype=np.int32)
        for t, l in zip(ts, ls):
            for x, d in zip(l, t.shape):
                dims[x] = d
    else:
        dims = _i32(label_dim)
    ranks = _i32([len(l) for l in ls])
    lab_ptrs = (ctypes.c_void_p * n)(*[l.ctypes.data for l in ls])
    dat_ptrs = (ctypes.c_void_p * n)(*[t.ctypes.data for t in ts])
    op = _i32(open_labels)
    pp = _i32([x for pr in path for x in pr])
    sl = _i32(list(sliced))
    num_slices = 1
    for l in sliced:
        num_slices *= int(dims[l])
    if slice_end is None:
        slice_end = num_slices
    out = np.zeros(tuple(int(dims[l]) for l in open_labels), dtype=np.complex128)
    rc = lib().orc_contract(n, ranks.ctypes.data, lab_ptrs, dat_ptrs, dims.ctypes.data,
                            len(dims), len(op), op.ctypes.data, len(path), pp.ctypes.data,
                            len(sl), sl.ctypes.data, int(slice_begin), int(slice_end),
                            out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_contract failed: %d" % rc)
    return out.reshape(-1)


def contract_network(net, path, sliced=(), slice_begin=0, slice_end=None):
    return contract(net.tensors, net.labels, net.open_labels, path, sliced, slice_begin,
                    slice_end)


def contract_sparse(tensors, labels, open_labels, path, samples):
    """Sparse-state contraction (Sec. 3.3): the amplitudes of the sampled bitstrings.

    ``samples`` is an (S, len(open_labels)) array of 0/1; column j is the value of
    open_labels[j].  Every tensor keeps, for the open labels it carries, only the configurations
    of those labels that occur among the samples (its merged sparse bond), each with a dense
    array over its other labels.  A pairwise step (path format of Sec. 3.1) takes the
    configurations of the union of its operands' open labels that occur among the samples; for
    each it picks the operand entries with the matching projections and contracts their dense
    parts with the plain einsum of Eq. chap2_einsum.  The root carries every open label and no
    dense label; entry i of the result is its value at sample i.  Every dense label must lie on
    exactly two tensors (no hyperedges)."""
    samples = np.asarray(samples, dtype=np.int64).reshape(-1, len(open_labels))
    col = {l: j for j, l in enumerate(open_labels)}

    def configs(open_ls):
        # distinct projections of the samples onto these open labels, sorted
        if not open_ls:
            return [()]
        cols = [col[l] for l in open_ls]
        return sorted(set(tuple(int(v) for v in row[cols]) for row in samples))

    items = []
    for t, ls in zip(tensors, labels):
        ls = [int(x) for x in ls]
        t = np.asarray(t, dtype=np.complex128)
        ol = sorted([l for l in ls if l in col], key=lambda l: col[l])
        dl = [l for l in ls if l not in col]
        vals = {}
        for cfg in configs(ol):
            at = dict(zip(ol, cfg))
            idx = tuple(at[l] if l in at else slice(None) for l in ls)
            vals[cfg] = np.ascontiguousarray(t[idx])  # dense labels in the tensor's order
        items.append((ol, dl, vals))
    last = 0
    for a, b in path:
        oa, da, va = items[a]
        ob, db, vb = items[b]
        oc = sorted(oa + ob, key=lambda l: col[l])
        shared = set(da) & set(db)
        dc = [l for l in da if l not in shared] + [l for l in db if l not in shared]
        vc = {}
        for cfg in configs(oc):
            at = dict(zip(oc, cfg))
            ca = tuple(at[l] for l in oa)
            cb = tuple(at[l] for l in ob)
            vc[cfg] = einsum_pair(va[ca], da, vb[cb], db, dc)
        items[a] = (oc, dc, vc)
        items[b] = None
        last = a
    oc, dc, vc = items[last]
    if dc or oc != list(open_labels):
        raise ValueError("the path does not reduce to the open labels")
    return np.array([complex(vc[tuple(int(v) for v in row)]) for row in samples],
                    dtype=np.complex128)


def statevector(n_qubits, gates):
    """Full 2^n state after ``gates`` (objects with .qubits and .matrix), qubit 0 = MSB."""
    g = len(gates)
    nq = _i32([len(x.qubits) for x in gates])
    q = np.zeros(2 * g, dtype=np.int32)
    m = np.zeros(16 * g, dtype=np.complex128)
    for i, x in enumerate(gates):
        for j, qq in enumerate(x.qubits):
            q[2 * i + j] = qq
        mm = np.asarray(x.matrix, dtype=np.complex128).reshape(-1)
        m[16 * i:16 * i + mm.size] = mm
    state = np.empty(1 << n_qubits, dtype=np.complex128)
    rc = lib().orc_statevector(n_qubits, g, nq.ctypes.data, q.ctypes.data, m.ctypes.data,
                               state.ctypes.data)
    if rc != 0:
        raise ValueError("orc_statevector failed: %d" % rc)
    return state


def readout(amps, n_qubits):
    """[sum p, sum p^2, F_l (Eq. lxeb_2), ideal-sample XEB 2^n sum p^2 / sum p - 1]."""
    a = np.ascontiguousarray(amps, dtype=np.complex128).reshape(-1)
    out = np.zeros(4, dtype=np.float64)
    rc = lib().orc_readout(a.size, a.ctypes.data, int(n_qubits), out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_readout failed: %d" % rc)
    return out


def rel_l2(a, ref):
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def eps_l2sq(a, ref):
    """Eq. (l2_squared_error): relative error of the squared L2 norm."""
    l2 = float(np.sum(np.abs(np.asarray(ref).reshape(-1)) ** 2))
    l2p = float(np.sum(np.abs(np.asarray(a).reshape(-1)) ** 2))
    return abs(l2 - l2p) / l2


def eps_f(eps_l2sq_value, F):
    """Eq. (lxeb_as_l2_error): relative error of F_l implied by eps_L2^2."""
    return eps_l2sq_value * (1.0 + F) / F
