"""Python binding of the C ABI in ``include/tn.h`` (libtn.so): argument marshalling only.

Every step of the contraction runs in libtn.so's CUDA kernels.  PyTorch supplies device memory
(amplitude buffers, optional workspace) and streams.  If libtn.so is missing this module raises;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtn.so")

TN_OK = 0
STATUS = {0: "TN_OK", 1: "TN_ERR_INVALID_ARG", 2: "TN_ERR_SHAPE", 3: "TN_ERR_PATH",
          4: "TN_ERR_OOM", 5: "TN_ERR_CUDA", 6: "TN_ERR_TIMEOUT", 7: "TN_ERR_UNSUPPORTED",
          8: "TN_ERR_NUMERIC"}
PRECISION = {"c64": 0, "tf32": 1, "split_tf32": 2, "fp16_scaled": 3, "bf16_scaled": 4,
             "split_bf16": 5, "split_fp16": 6, "mixed": 7}
GEMM_FORM = {"auto": 0, "4m": 1, "3m": 2}
KERNELS = {0: "generic", 1: "stream", 2: "gemm_simt", 3: "gemm_tc", 4: "thin_tc"}

# Every symbol declared in include/tn.h.
EXPORTS = ("tn_network_load", "tn_network_set_data", "tn_plan", "tn_plan_get_info",
           "tn_plan_get_step_info", "tn_contract", "tn_contract_host", "tn_readout",
           "tn_readout_noalloc", "tn_selftest_wait_timeout", "tn_path_optimize",
           "tn_sparse_plan", "tn_sparse_contract", "tn_sparse_get_info", "tn_destroy",
           "tn_status_string", "tn_last_error_detail")


class PlanOptions(C.Structure):
    _fields_ = [("max_slices_in_flight", C.c_int64), ("workspace_limit", C.c_int64),
                ("workspace", C.c_void_p), ("gemm_form", C.c_int32),
                ("sync_each_call", C.c_int32), ("use_graph", C.c_int32),
                ("profile", C.c_int32), ("tc_bk", C.c_int32), ("tc_bn", C.c_int32),
                ("autotune", C.c_int32), ("mixed_topk", C.c_int32), ("thin_tc", C.c_int32),
                ("eps_budget", C.c_double), ("reserved", C.c_int32 * 2)]


class PlanInfo(C.Structure):
    _fields_ = [("num_steps", C.c_int64), ("num_slices", C.c_int64),
                ("slices_in_flight", C.c_int64), ("workspace_bytes", C.c_int64),
                ("num_open", C.c_int32), ("max_log2_size", C.c_int32),
                ("tcc_per_slice", C.c_double), ("tcc_invariant", C.c_double),
                ("tmc_per_slice", C.c_double), ("num_tc_steps", C.c_int32),
                ("num_gemm_steps", C.c_int32), ("num_stream_steps", C.c_int32),
                ("num_generic_steps", C.c_int32), ("kernel_launches", C.c_int64),
                ("bind_ms", C.c_double), ("bind_launches", C.c_int64),
                ("num_single_pass", C.c_int32), ("num_compensated", C.c_int32),
                ("eps_predicted", C.c_double), ("num_open_sliced", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class StepInfo(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("slice_dependent", C.c_int32), ("log2_m", C.c_int32),
                ("log2_n", C.c_int32), ("log2_k", C.c_int32), ("log2_batch", C.c_int32),
                ("log2_a", C.c_int32), ("log2_b", C.c_int32), ("log2_c", C.c_int32),
                ("gemm_form", C.c_int32), ("tcc", C.c_double), ("time_ms", C.c_double),
                ("launches", C.c_int64), ("prep_ms", C.c_double), ("tc_variant", C.c_int32),
                ("store_run_log2", C.c_int32), ("tmc_bytes", C.c_double)]


class PathOptions(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("sweeps", C.c_int32), ("sweeps_per_slice", C.c_int32),
                ("sweeps_final", C.c_int32), ("max_log2_size", C.c_int32),
                ("max_sliced", C.c_int32), ("chains", C.c_int32), ("t_start", C.c_double),
                ("t_end", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("greedy_trials", C.c_int32), ("balance_log2", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class PathInfo(C.Structure):
    _fields_ = [("log2_tcc", C.c_double), ("log2_tcc_total", C.c_double),
                ("log2_tmc", C.c_double), ("score", C.c_double),
                ("initial_log2_tcc", C.c_double), ("initial_max_log2_size", C.c_int32),
                ("max_log2_size", C.c_int32), ("num_sliced", C.c_int32),
                ("reserved0", C.c_int32), ("moves_tried", C.c_int64),
                ("moves_accepted", C.c_int64), ("reserved", C.c_int64 * 4)]


class SparseInfo(C.Structure):
    _fields_ = [("num_steps", C.c_int64), ("num_samples", C.c_int64),
                ("distinct_samples", C.c_int64), ("total_configs", C.c_int64),
                ("arena_bytes", C.c_int64), ("tcc", C.c_double), ("kernel_launches", C.c_int64),
                ("max_log2_dense", C.c_int32), ("gemm_steps", C.c_int32),
                ("dense_subtrees", C.c_int64), ("dense_subtree_steps", C.c_int64),
                ("thin_steps", C.c_int64), ("grouped_steps", C.c_int64)]


class TnError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__("%s: %s" % (STATUS.get(status, status), detail))
        self.status = status
        self.detail = detail


_lib = None


def lib():
    """Load libtn.so (built by ``__graft_entry__.build()``); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtn.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.tn_network_load.argtypes = [i32, vp, vp, vp, vp, i32, vp, C.POINTER(vp)]
        L.tn_network_set_data.argtypes = [vp, vp]
        L.tn_plan.argtypes = [vp, i32, vp, i32, vp, C.c_int, C.POINTER(PlanOptions),
                              C.POINTER(vp)]
        L.tn_plan_get_info.argtypes = [vp, C.POINTER(PlanInfo)]
        L.tn_plan_get_step_info.argtypes = [vp, i64, C.POINTER(StepInfo)]
        L.tn_contract.argtypes = [vp, i64, i64, vp, vp]
        L.tn_contract_host.argtypes = [vp, i64, i64, vp, vp]
        L.tn_readout.argtypes = [vp, vp, i32, vp, vp]
        L.tn_readout_noalloc.argtypes = [vp, i64, i32, vp, vp]
        L.tn_selftest_wait_timeout.argtypes = [i32, vp]
        L.tn_path_optimize.argtypes = [i32, vp, vp, i32, vp, vp, C.POINTER(PathOptions), vp, vp,
                                       i32, C.POINTER(PathInfo)]
        L.tn_sparse_plan.argtypes = [vp, i32, vp, i64, vp, C.c_int, C.POINTER(vp)]
        L.tn_sparse_contract.argtypes = [vp, vp, vp]
        L.tn_sparse_get_info.argtypes = [vp, C.POINTER(SparseInfo)]
        L.tn_destroy.argtypes = [vp]
        L.tn_destroy.restype = None
        L.tn_status_string.argtypes = [C.c_int]
        L.tn_status_string.restype = C.c_char_p
        L.tn_last_error_detail.argtypes = [vp, C.c_size_t]
        for name in EXPORTS:
            if name not in ("tn_destroy", "tn_status_string"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status):
    if status != TN_OK:
        buf = C.create_string_buffer(1024)
        lib().tn_last_error_detail(buf, 1024)
        raise TnError(status, buf.value.decode(errors="replace"))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _device_amps(amps, numel=None, what="amps"):
    """Check that ``amps`` is a contiguous complex128 CUDA tensor (of ``numel`` entries when
    given) before its address goes to a kernel: the kernels read or write numel complex128
    values at that address, so another dtype, a host tensor or a strided view would send them
    past the buffer."""
    import torch
    if not isinstance(amps, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % what)
    if amps.dtype != torch.complex128:
        raise TypeError("%s must be complex128, got %s" % (what, amps.dtype))
    if not amps.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if numel is not None and amps.numel() != numel:
        raise ValueError("%s must have %d entries, got %d" % (what, numel, amps.numel()))
    if numel is None and amps.numel() == 0:
        raise ValueError("%s is empty" % what)
    if not amps.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    return C.c_void_p(amps.data_ptr())


def readout_noalloc(amps, n_qubits, stream=None):
    """FP64 readout of a complex128 CUDA tensor without a plan and without device allocation
    (tn_readout_noalloc): [sum p, sum p^2, F_l, ideal-sample XEB]."""
    out = np.zeros(4, dtype=np.float64)
    ptr = _device_amps(amps)
    _check(lib().tn_readout_noalloc(ptr, int(amps.numel()),
                                    int(n_qubits), C.c_void_p(out.ctypes.data),
                                    _stream_ptr(stream)))
    return out


def path_optimize(labels, open_labels, path, seed=0, sweeps=-1, sweeps_per_slice=-1,
                  sweeps_final=-1, max_log2_size=0, max_sliced=0, chains=1, t_start=0.0,
                  t_end=0.0, alpha=0.0, beta=0.0, greedy_trials=0, balance_log2=0):
    """Simulated-annealing path optimisation with dynamic slicing (tn_path_optimize, host
    only).  ``labels`` per tensor, ``open_labels`` the output labels, ``path`` the starting
    pairs; ``balance_log2`` > 0 weighs the multiply-adds of unbalanced steps (k < 64 or
    min(m, n) < 32 as a GEMM) 2^balance_log2 times in the score.  Returns (path, sliced_labels,
    info dict)."""
    n = len(labels)
    ranks = np.array([len(l) for l in labels], dtype=np.int32)
    labs = [np.ascontiguousarray(np.asarray(l, dtype=np.int32)) for l in labels]
    lab_p = (C.c_void_p * n)(*[l.ctypes.data if len(l) else None for l in labs])
    op = np.ascontiguousarray(np.asarray(open_labels, dtype=np.int32))
    pin = np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1))
    if pin.size != 2 * (n - 1):
        raise ValueError("path must have num_tensors - 1 pairs")
    pout = np.zeros(max(1, 2 * (n - 1)), dtype=np.int32)
    cap = 64
    sl = np.zeros(cap, dtype=np.int32)
    o = PathOptions(seed=seed, sweeps=sweeps, sweeps_per_slice=sweeps_per_slice,
                    sweeps_final=sweeps_final, max_log2_size=max_log2_size,
                    max_sliced=max_sliced, chains=chains, t_start=t_start, t_end=t_end,
                    alpha=alpha, beta=beta, greedy_trials=greedy_trials,
                    balance_log2=balance_log2)
    info = PathInfo()
    _check(lib().tn_path_optimize(n, ranks.ctypes.data, lab_p, len(op),
                                  op.ctypes.data if len(op) else None,
                                  pin.ctypes.data if pin.size else None, C.byref(o),
                                  pout.ctypes.data, sl.ctypes.data, cap, C.byref(info)))
    pairs = [(int(pout[2 * i]), int(pout[2 * i + 1])) for i in range(n - 1)]
    d = {f: getattr(info, f) for f, _ in PathInfo._fields_ if not f.startswith("reserved")}
    return pairs, [int(x) for x in sl[:info.num_sliced]], d


class Network:
    """A tensor network on the device (tn_network_load)."""

    def __init__(self, tensors, labels, open_labels):
        self._keep = []
        n = len(tensors)
        # np.array keeps rank-0 tensors 0-d (np.ascontiguousarray would make them 1-d)
        arrs = [np.array(t, dtype=np.complex128, order="C") for t in tensors]
        ranks = np.array([a.ndim for a in arrs], dtype=np.int32)
        labs = [np.ascontiguousarray(np.asarray(l, dtype=np.int32).reshape(-1)) for l in labels]
        if len(labels) != n or any(len(l) != a.ndim for l, a in zip(labs, arrs)):
            raise ValueError("every tensor needs one label per axis")
        dims = [np.ascontiguousarray(np.asarray(a.shape, dtype=np.int64)) for a in arrs]
        lab_p = (C.c_void_p * n)(*[l.ctypes.data for l in labs])
        dim_p = (C.c_void_p * n)(*[d.ctypes.data for d in dims])
        dat_p = (C.c_void_p * n)(*[a.ctypes.data for a in arrs])
        op = np.ascontiguousarray(np.asarray(open_labels, dtype=np.int32))
        h = C.c_void_p()
        _check(lib().tn_network_load(n, ranks.ctypes.data, lab_p, dim_p, dat_p, len(op),
                                     op.ctypes.data if len(op) else None, C.byref(h)))
        self.handle = h
        self.num_tensors = n
        self.num_open = len(op)
        self.data_bytes = sum(a.nbytes for a in arrs)

    @classmethod
    def from_workload(cls, net):
        return cls(net.tensors, net.labels, net.open_labels)

    def set_data(self, tensors):
        arrs = [np.array(t, dtype=np.complex128, order="C") for t in tensors]
        dat_p = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        _check(lib().tn_network_set_data(self.handle, dat_p))

    def close(self):
        if self.handle:
            lib().tn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """An execution plan (tn_plan) over a Network."""

    def __init__(self, network: Network, path, sliced=(), mode="c64", max_slices_in_flight=0,
                 workspace_limit=0, workspace=None, gemm_form="auto", sync_each_call=False,
                 profile=False, use_graph=False, tc_bk=0, tc_bn=0, autotune=False,
                 mixed_topk=0, eps_budget=0.0, thin_tc=0):
        self.network = network
        opts = PlanOptions()
        opts.max_slices_in_flight = int(max_slices_in_flight)
        opts.workspace_limit = int(workspace_limit)
        self._workspace = workspace  # a torch tensor kept alive by the plan
        if workspace is not None:
            opts.workspace = C.c_void_p(workspace.data_ptr())
            opts.workspace_limit = int(workspace.numel() * workspace.element_size())
        opts.gemm_form = GEMM_FORM[gemm_form]
        opts.sync_each_call = 1 if sync_each_call else 0
        opts.profile = 1 if profile else 0
        opts.use_graph = 1 if use_graph else 0
        opts.tc_bk = int(tc_bk)
        opts.tc_bn = int(tc_bn)
        opts.autotune = 1 if autotune else 0
        opts.mixed_topk = int(mixed_topk)
        opts.eps_budget = float(eps_budget)
        opts.thin_tc = int(thin_tc)
        pp = np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1))
        sl = np.ascontiguousarray(np.asarray(list(sliced), dtype=np.int32))
        h = C.c_void_p()
        _check(lib().tn_plan(network.handle, len(path), pp.ctypes.data if pp.size else None,
                             len(sl), sl.ctypes.data if sl.size else None, PRECISION[mode],
                             C.byref(opts), C.byref(h)))
        self.handle = h
        self.mode = mode

    def info(self) -> dict:
        i = PlanInfo()
        _check(lib().tn_plan_get_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in PlanInfo._fields_ if not f.startswith("reserved")}

    def step_info(self, step: int) -> dict:
        s = StepInfo()
        _check(lib().tn_plan_get_step_info(self.handle, int(step), C.byref(s)))
        d = {f: getattr(s, f) for f, _ in StepInfo._fields_ if not f.startswith("reserved")}
        d["kernel_name"] = KERNELS.get(d["kernel"], "?")
        return d

    def contract(self, amps, slice_begin=0, slice_end=None, stream=None):
        """amps: torch complex128 CUDA tensor of 2^num_open entries; results are added."""
        if slice_end is None:
            slice_end = self.info()["num_slices"]
        ptr = _device_amps(amps, 1 << self.network.num_open)
        _check(lib().tn_contract(self.handle, int(slice_begin), int(slice_end), ptr,
                                 _stream_ptr(stream)))

    def contract_host(self, slice_begin=0, slice_end=None, stream=None, out=None):
        """Contract into a host complex128 numpy array (synchronises)."""
        if slice_end is None:
            slice_end = self.info()["num_slices"]
        n = 1 << self.network.num_open
        if out is None:
            out = np.zeros(n, dtype=np.complex128)
        if (not isinstance(out, np.ndarray) or out.dtype != np.complex128 or out.size != n
                or not out.flags.c_contiguous):
            raise ValueError("out must be a contiguous complex128 array of %d entries" % n)
        _check(lib().tn_contract_host(self.handle, int(slice_begin), int(slice_end),
                                      C.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def readout(self, amps, n_qubits, stream=None):
        out = np.zeros(4, dtype=np.float64)
        ptr = _device_amps(amps, 1 << self.network.num_open)
        _check(lib().tn_readout(self.handle, ptr, int(n_qubits),
                                C.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def close(self):
        if self.handle:
            lib().tn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SparsePlan:
    """Sparse-state contraction of a network for a list of sampled bitstrings (tn_sparse_plan;
    Sec. 3.3).  ``samples``: (S, num_open) array of 0/1, column j = open label j."""

    def __init__(self, network, path, samples, mode="c64"):
        self.network = network
        smp = np.ascontiguousarray(np.asarray(samples, dtype=np.uint8))
        if smp.ndim != 2 or smp.shape[1] != network.num_open:
            raise ValueError("samples must be (S, num_open)")
        self.num_samples = smp.shape[0]
        pp = np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1))
        h = C.c_void_p()
        _check(lib().tn_sparse_plan(network.handle, len(pp) // 2,
                                    pp.ctypes.data if pp.size else None, smp.shape[0],
                                    smp.ctypes.data, PRECISION[mode], C.byref(h)))
        self.handle = h

    def contract(self, amps, stream=None):
        """ADD the samples' amplitudes into a complex128 CUDA tensor of num_samples entries."""
        ptr = _device_amps(amps, self.num_samples)
        _check(lib().tn_sparse_contract(self.handle, ptr, _stream_ptr(stream)))

    def info(self):
        i = SparseInfo()
        _check(lib().tn_sparse_get_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in SparseInfo._fields_ if not f.startswith("reserved")}

    def close(self):
        if self.handle:
            lib().tn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
