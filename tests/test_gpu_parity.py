"""GPU path (through the C ABI) against the CPU oracle, element by element.

Tolerances (amplitude relative L2 error against FP64, and the same bound per entry relative
to the largest reference amplitude: max |a - a_ref| <= tol * max |a_ref|):
  complex64 path            <= 1e-5
  FP16 / BF16 scaled path   <= 5e-3 (BF16: the precision policy keeps single-pass BF16 on as
                               many of the largest dense steps as fit that bar, the others
                               compensated)
  compensated FP16 / BF16   <= 1e-5 / 1e-4 (hi + lo operand planes, three products)
  TF32 / 3xTF32             <= 5e-3 / 1e-5 (10-bit significand like FP16; hi + lo as above)
and for the full-size circuit the ideal-sample XEB (2^n sum p^2 / sum p - 1) within 1e-3
relative of the state-vector value in every mode.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_03978_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# split_fp16: hi + lo hold ~22 significant bits and the dropped lo*lo term is ~2^-22; with the
# accumulator promoted every 512 of K a single step stays near 4e-6 (any K), so single steps are
# held to the complex64 bar; a whole circuit adds ~7 such steps and its FP32 steps, hence 5e-5
# there (CIRCUIT_TOL).  split_bf16: ~2^-16 per product.  mixed: bounded by its FP16 steps.
TOL = {"c64": 1e-5, "fp16_scaled": 5e-3, "bf16_scaled": 5e-3, "split_fp16": 1e-5,
       "split_bf16": 1e-4, "mixed": 5e-3, "tf32": 5e-3, "split_tf32": 1e-5}
CIRCUIT_TOL = dict(TOL, split_fp16=5e-5, split_tf32=5e-5)


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_03978_gb300 import tn as T
    T.lib()
    return T


def crandn(rng, rank, scale=1.0):
    shape = (2,) * rank
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale


def gpu_amps(tn, tensors, labels, open_labels, path, sliced=(), mode="c64", s0=0, s1=None,
             **kw):
    net = tn.Network(tensors, labels, open_labels)
    plan = tn.Plan(net, path, sliced, mode=mode, sync_each_call=True, **kw)
    amps = torch.zeros(1 << len(open_labels), dtype=torch.complex128, device="cuda")
    plan.contract(amps, s0, s1)
    torch.cuda.synchronize()
    out = amps.cpu().numpy()
    info = plan.info()
    kernels = [plan.step_info(i)["kernel_name"] for i in range(info["num_steps"])]
    plan.close()
    net.close()
    return out, info, kernels


def read_golden(name):
    rows = np.loadtxt(os.path.join(HERE, "golden", name + ".amps.txt"), comments="#")
    return rows[:, 0] + 1j * rows[:, 1]


def check(got, ref, tol):
    got, ref = np.asarray(got).reshape(-1), np.asarray(ref).reshape(-1)
    err = O.rel_l2(got, ref)
    assert err <= tol, "rel L2 %.3e > %.1e" % (err, tol)
    # per entry: no amplitude may be off by more than tol of the largest one (a few badly wrong
    # small amplitudes would hide inside the L2 norm)
    worst = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert worst <= tol, "max |delta a| / max |a| %.3e > %.1e" % (worst, tol)
    return err


# ------------------------------------------------------------------ whole circuits
@pytest.mark.parametrize("mode", ["c64", "fp16_scaled", "bf16_scaled"])
def test_small_circuit_vs_oracle_and_statevector(tn, mode):
    wl = W.small_workload()
    net = wl.network
    ref = O.contract_network(net, wl.path)
    got, info, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, mode=mode)
    check(got, ref, TOL[mode])
    check(got, read_golden("sycamore_3x4_c8_open6"), TOL[mode])
    assert info["num_slices"] == 1


def test_closed_forms(tn):
    n = 10
    net = W.build_network(W.hadamard_circuit(n), list(range(n)), {})
    got, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels,
                         W.greedy_path(net.labels, net.open_labels))
    check(got, np.full(1 << n, 2 ** (-n / 2)), TOL["c64"])
    net = W.build_network(W.ghz_circuit(n), list(range(n)), {})
    got, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels,
                         W.greedy_path(net.labels, net.open_labels))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 2 ** -0.5
    check(got, ref, TOL["c64"])
    circ = W.mirrored_circuit(W.random_circuit(3, 3, 5, seed=4))
    net = W.build_network(circ, list(range(9)), {})
    got, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels,
                         W.greedy_path(net.labels, net.open_labels))
    ref = np.zeros(1 << 9, dtype=complex)
    ref[0] = 1
    check(got, ref, TOL["c64"])


def test_slices_sum_to_unsliced_and_ranges_split(tn):
    wl = W.small_workload()
    net = wl.network
    sl = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    ref = O.contract_network(net, wl.path)
    full, info, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, sl)
    assert info["num_slices"] == 8
    check(full, ref, 1e-5)
    a, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, sl, s0=0, s1=3)
    b, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, sl, s0=3, s1=8)
    check(a + b, ref, 1e-5)
    check(a, O.contract_network(net, wl.path, sl, 0, 3), 1e-5)
    # one slice per launch gives the same sum
    one, info1, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, sl,
                             max_slices_in_flight=1)
    assert info1["slices_in_flight"] == 1
    check(one, full, 1e-6)


def test_degenerate_networks_and_ragged_batches(tn):
    rng = np.random.default_rng(77)
    # a single tensor (no pairwise step): the amplitudes are the tensor in the open order
    T = crandn(rng, 6)
    lab = [5, 3, 1, 0, 4, 2]
    out = [0, 1, 2, 3, 4, 5]
    got, info, _ = gpu_amps(tn, [T], [lab], out, [])
    assert info["num_steps"] == 0
    check(got, np.transpose(T, [lab.index(l) for l in out]).reshape(-1), 1e-6)
    # no open label: the contraction is a scalar
    A, B = crandn(rng, 5), crandn(rng, 5)
    la = [10, 11, 12, 13, 14]
    lb = [14, 12, 10, 13, 11]
    got, _, _ = gpu_amps(tn, [A, B], [la, lb], [], [(0, 1)])
    check(got, O.contract([A, B], [la, lb], [], [(0, 1)]), 1e-5)
    # an empty slice range adds nothing; 8 slices in batches of 3, 3, 2
    wl = W.small_workload()
    net = wl.network
    sl = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    ref = O.contract_network(net, wl.path)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.Plan(tnet, wl.path, sl, mode="c64", max_slices_in_flight=3, sync_each_call=True)
    amps = torch.zeros(1 << len(net.open_labels), dtype=torch.complex128, device="cuda")
    plan.contract(amps, 2, 2)
    assert torch.count_nonzero(amps).item() == 0
    assert plan.info()["slices_in_flight"] == 3
    plan.contract(amps)
    torch.cuda.synchronize()
    check(amps.cpu().numpy(), ref, 1e-5)
    with pytest.raises(tn.TnError):
        plan.contract(amps, 0, 9)  # past the last slice
    plan.close()
    tnet.close()


def test_all_open_norm_and_readout(tn):
    circ = W.random_circuit(3, 4, 10, seed=8)
    net = W.build_network(circ, list(range(12)), {})
    path = W.greedy_path(net.labels, net.open_labels)
    ref = O.statevector(12, circ.gates)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.Plan(tnet, path, (), mode="c64", sync_each_call=True)
    amps = torch.zeros(1 << 12, dtype=torch.complex128, device="cuda")
    plan.contract(amps)
    got = amps.cpu().numpy()
    check(got, ref, 1e-5)
    r_gpu = plan.readout(amps, 12)
    r_cpu = O.readout(got, 12)
    np.testing.assert_allclose(r_gpu, r_cpu, rtol=1e-12, atol=1e-12)
    assert abs(r_gpu[0] - 1) < 1e-5
    plan.close()
    tnet.close()


# ------------------------------------------------------------------ single steps per kernel
def single_step(rng, lm, ln, lk, scale=1.0, scramble=True):
    M = list(range(0, lm))
    N = list(range(100, 100 + ln))
    K = list(range(200, 200 + lk))
    la = list(rng.permutation(M + K))
    lb = list(rng.permutation(N + K))
    out = M + N
    if scramble:
        out = list(rng.permutation(out))
    A = crandn(rng, lm + lk, scale)
    B = crandn(rng, ln + lk, scale)
    return [A, B], [[int(x) for x in la], [int(x) for x in lb]], [int(x) for x in out]


@pytest.mark.parametrize("shape,kernel", [
    ((3, 2, 2), "generic"),      # tiny
    ((9, 9, 1), "generic"),      # outer-product-like: 2^18 outputs, k = 2
    ((9, 9, 2), "gemm_simt"),    # k = 4: register-tiled, zero-padded K tile
    ((2, 2, 9), "generic"),      # 16 outputs of 512 terms each
    ((2, 2, 11), "gemm_simt"),   # k >= 2^10 into a small result: split along K
    ((10, 1, 13), "gemm_simt"),  # a 2-wide result of a long contraction
    ((6, 5, 4), "gemm_simt"),
    ((7, 6, 9), "gemm_simt"),
    ((5, 9, 4), "gemm_simt"),
    ((6, 4, 14), "gemm_simt"),   # few outputs, long contraction: split along K
    ((3, 3, 13), "gemm_simt"),
    ((5, 5, 13), "gemm_simt"),   # 32 x 32 result, long contraction: the skinny split-K form
    ((5, 5, 16), "gemm_simt"),
])
def test_single_step_cuda_core_kernels(tn, shape, kernel):
    rng = np.random.default_rng(sum(shape))
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)])
    assert kernels == [kernel]
    check(got, ref, 1e-5)
    # the same step with 4 slices in flight (a sliced bond on a rank-1 factor of A)
    A, B = tensors
    v = crandn(rng, 1)
    t2 = [A[None] * v.reshape(2, *([1] * A.ndim)), B, np.ones(2, complex)]
    l2 = [[900] + labels[0], labels[1], [900]]
    ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
    got2, info, _ = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900])
    assert info["slices_in_flight"] == 2
    check(got2, ref2, 1e-5)


def test_long_contraction_with_a_batch_label_on_the_elementwise_kernel(tn):
    # a hyperedge b on three tensors is a batch index of the step that meets two of them; such
    # steps run element-wise, here with k = 2^11 (offsets computed without the shared table)
    rng = np.random.default_rng(66)
    K = list(range(200, 211))
    tensors = [crandn(rng, 14, 2.0 ** -6), crandn(rng, 13, 2.0 ** -6), crandn(rng, 1)]
    labels = [[500] + K + [0, 1], [500] + K + [100], [500]]
    out = [100, 0, 1]
    path = [(0, 1), (0, 2)]
    ref = O.contract(tensors, labels, out, path)
    got, _, kernels = gpu_amps(tn, tensors, labels, out, path)
    assert kernels[0] == "generic"
    check(got, ref, 1e-5)


@pytest.mark.parametrize("shape", [(12, 6, 0), (14, 2, 0), (3, 12, 0), (10, 0, 0)])
def test_outer_product_steps(tn, shape):
    # nothing contracted (an outer product; C's order scrambled): the element-wise kernel's
    # store-stream path, one slice and 2 slices in flight, and with a batch label (a hyperedge
    # that two operands and a third tensor share)
    rng = np.random.default_rng(600 + 3 * shape[0] + 5 * shape[1])
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)])
    assert kernels == ["generic"]
    check(got, ref, 1e-5)
    A, B = tensors
    v = crandn(rng, 1)
    t2 = [A[None] * v.reshape(2, *([1] * A.ndim)), B, np.ones(2, complex)]
    l2 = [[900] + labels[0], labels[1], [900]]
    ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
    for mode in ("c64", "fp16_scaled"):
        got2, info, k2 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode=mode)
        assert info["slices_in_flight"] == 2 and k2[0] == "generic"
        check(got2, ref2, 1e-5)
    # a batch label b on A, B and a vector: C[b, m, n] = A[b, m] B[b, n], then summed over b
    w = crandn(rng, 1)
    t3 = [A[None] * v.reshape(2, *([1] * A.ndim)), B[None] * w.reshape(2, *([1] * B.ndim)),
          crandn(rng, 1)]
    l3 = [[950] + labels[0], [950] + labels[1], [950]]
    ref3 = O.contract(t3, l3, out, [(0, 1), (0, 2)])
    got3, _, k3 = gpu_amps(tn, t3, l3, out, [(0, 1), (0, 2)])
    assert k3[0] == "generic"
    check(got3, ref3, 1e-5)


@pytest.mark.parametrize("shape", [(12, 4, 4), (10, 2, 6), (4, 11, 3), (13, 0, 2), (11, 3, 1),
                                   (1, 12, 5), (14, 2, 2), (12, 1, 3), (10, 4, 1), (18, 2, 2),
                                   (3, 17, 1), (12, 3, 8), (10, 4, 10), (3, 13, 9), (11, 0, 7)])
def test_thin_steps_stream_kernel(tn, shape):
    # a contraction (k <= 1024) of a large operand with one of at most 16 free elements: one
    # thread per row of the large operand (the small one may be either side); k <= 8 loads rows
    # into registers, longer k stages them in shared memory (the small operand 64 of k at a
    # time); 2 slices in flight too
    rng = np.random.default_rng(500 + 3 * shape[0] + 5 * shape[1] + shape[2])
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)])
    assert kernels == ["stream"]
    check(got, ref, 1e-5)
    A, B = tensors
    v = crandn(rng, 1)
    t2 = [A[None] * v.reshape(2, *([1] * A.ndim)), B, np.ones(2, complex)]
    l2 = [[900] + labels[0], labels[1], [900]]
    ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
    for mode in ("c64", "fp16_scaled"):
        got2, info, k2 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode=mode)
        assert info["slices_in_flight"] == 2 and k2[0] == thin_kernel(shape, mode)
        check(got2, ref2, 1e-5)


def thin_kernel(shape, mode, thin_tc=0):
    """The kernel a slice-dependent streaming step of GEMM extents (lm, ln, lk) runs on: the
    tensor cores in the tensor-core modes for 4-16 columns and 4-16 terms (by default with 16
    terms, or 16 columns and 8 terms), else the CUDA cores."""
    lm, ln, lk = shape
    wide, narrow = max(lm, ln), min(lm, ln)
    fits = 8 <= wide <= 30 and 2 <= narrow <= 4 and 2 <= lk <= 4
    on = thin_tc > 0 or (thin_tc == 0 and (lk == 4 or (narrow == 4 and lk == 3)))
    return "thin_tc" if mode != "c64" and fits and on else "stream"


# (lm, ln, lk): every column / term count of the tensor-core thin kernel, the small operand on
# either side, 4 tiles (2^10 rows) up to a ragged multiple of the SM count of tiles
THIN_TC_SHAPES = [(12, 2, 2), (11, 2, 3), (13, 2, 4), (12, 3, 2), (3, 12, 3), (12, 3, 4),
                  (12, 4, 2), (11, 4, 3), (4, 12, 4), (10, 4, 4), (16, 4, 4), (17, 3, 3)]


@pytest.mark.parametrize("shape", THIN_TC_SHAPES)
def test_thin_steps_on_the_tensor_cores(tn, shape):
    # the streaming step as one real TF32 product with compensated operands (Sec. 4.2's 3xTF32):
    # FP32-level accuracy against the oracle, one slice and 2 slices in flight (the large
    # operand sliced; the small one sliced too); the CUDA-core form of the same step agrees
    rng = np.random.default_rng(700 + 3 * shape[0] + 5 * shape[1] + shape[2])
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    A, B = tensors
    v = crandn(rng, 1)
    big = 0 if shape[0] >= shape[1] else 1
    t2 = [A, B, np.ones(2, complex)]
    t2[big] = tensors[big][None] * v.reshape(2, *([1] * tensors[big].ndim))
    l2 = [list(labels[0]), list(labels[1]), [900]]
    l2[big] = [900] + l2[big]
    ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
    # both operands sliced: the small one varies with the slice too
    w = crandn(rng, 1)
    t3 = list(t2)
    t3[1 - big] = tensors[1 - big][None] * w.reshape(2, *([1] * tensors[1 - big].ndim))
    l3 = [list(l2[0]), list(l2[1]), [900]]
    l3[1 - big] = [900] + l3[1 - big]
    ref3 = O.contract(t3, l3, out, [(0, 1), (0, 2)])
    for mode in ("fp16_scaled", "tf32"):
        for flag in (1, -1):
            kind = "thin_tc" if flag > 0 else "stream"
            got2, info, k2 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode=mode,
                                      thin_tc=flag)
            assert info["slices_in_flight"] == 2 and k2[0] == kind
            check(got2, ref2, 1e-5)
            got3, _, k3 = gpu_amps(tn, t3, l3, out, [(0, 1), (0, 2)], [900], mode=mode,
                                   thin_tc=flag)
            assert k3[0] == kind
            check(got3, ref3, 1e-5)
        # the automatic choice
        _, _, k4 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode=mode)
        assert k4[0] == thin_kernel(shape, mode)
    # the complex64 mode keeps the CUDA cores whatever the option says
    _, _, k5 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode="c64", thin_tc=1)
    assert k5[0] == "stream"


@pytest.mark.parametrize("shape", [(19, 4, 3), (20, 4, 4), (19, 2, 2)])
@pytest.mark.parametrize("cfg", ["A", "B", "AB"])
def test_thin_tensor_core_slices_and_many_tiles(tn, shape, cfg):
    # 4 slices in flight (two sliced labels) on the large operand, the small one or both, with
    # 2^11-2^12 tiles per slice, so every CTA walks dozens of tiles (the raw ring, the hi / lo
    # slots and both accumulator buffers are reused many times): against the oracle, and the
    # same result bit for bit on a second call
    lm, ln, lk = shape
    rng = np.random.default_rng(800 + 7 * lm + 3 * ln + lk + len(cfg))
    M, N, K = list(range(0, lm)), list(range(100, 100 + ln)), list(range(200, 200 + lk))
    t = [crandn(rng, lm + lk), crandn(rng, ln + lk)]
    lab = [[int(x) for x in rng.permutation(M + K)], [int(x) for x in rng.permutation(N + K)]]
    extra = [900, 901]
    for x in extra:
        for side in (0, 1):
            if "AB"[side] in cfg:
                v = crandn(rng, 1)
                t[side] = t[side][None] * v.reshape(2, *([1] * t[side].ndim))
                lab[side] = [x] + lab[side]
    tensors = t + [np.ones(2, complex) for _ in extra]
    labels = lab + [[x] for x in extra]
    out = [int(x) for x in rng.permutation(M + N)]
    path = [(0, 1)] + [(0, 2 + j) for j in range(len(extra))]
    ref = O.contract(tensors, labels, out, path)
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, path, extra, mode="fp16_scaled", sync_each_call=True, thin_tc=1)
    assert plan.step_info(0)["kernel_name"] == "thin_tc" and plan.info()["slices_in_flight"] == 4
    first = plan.contract_host()
    check(first, ref, 1e-5)
    assert np.array_equal(plan.contract_host(), first)
    plan.close()
    net.close()


def test_thin_tensor_core_falls_back_when_c_order_leaves_the_tile(tn):
    # the tensor-core thin kernel takes 128-row tiles and needs C's three lowest positions inside
    # a tile; when a result order puts row bit 7 there the step runs on the CUDA cores (256-row
    # tiles) instead.  Seeded result orders are tried until both cases occur; both agree with the
    # oracle
    seen = set()
    for seed in range(60):
        rng = np.random.default_rng(4000 + seed)
        tensors, labels, out = single_step(rng, 12, 4, 4)
        ref = O.contract(tensors, labels, out, [(0, 1)])
        A, B = tensors
        v = crandn(rng, 1)
        t2 = [A[None] * v.reshape(2, *([1] * A.ndim)), B, np.ones(2, complex)]
        l2 = [[900] + labels[0], labels[1], [900]]
        ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
        got, _, k = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode="fp16_scaled",
                             thin_tc=1)
        check(got, ref2, 1e-5)
        seen.add(k[0])
        if seen == {"thin_tc", "stream"}:
            break
    assert "thin_tc" in seen
    if "stream" not in seen:
        pytest.skip("no seeded result order put row bit 7 among C's lowest three positions")


def test_thin_tensor_core_step_far_magnitudes(tn):
    # operands near 2^-60 and 2^+40 (FP32 range, far from 1): the hi / lo split is relative, so
    # the compensated products keep their accuracy at any scale
    rng = np.random.default_rng(777)
    for sa, sb in ((2.0 ** -60, 2.0 ** -50), (2.0 ** 40, 2.0 ** -30)):
        tensors, labels, out = single_step(rng, 14, 4, 4)
        tensors = [tensors[0] * sa, tensors[1] * sb]
        v = crandn(rng, 1)
        t2 = [tensors[0][None] * v.reshape(2, *([1] * tensors[0].ndim)), tensors[1],
              np.ones(2, complex)]
        l2 = [[900] + labels[0], labels[1], [900]]
        ref = O.contract(t2, l2, out, [(0, 1), (0, 2)])
        got, _, k = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode="fp16_scaled",
                             thin_tc=1)
        assert k[0] == "thin_tc"
        check(got, ref, 1e-5)


# (form, K-tile preference, N-tile preference): every tensor-core kernel variant
TC_VARIANTS = [("4m", 0, 0), ("4m", 64, 0), ("4m", 32, 0), ("4m", 0, 256), ("3m", 32, 0),
               ("3m", 64, 0)]


@pytest.mark.parametrize("form,bk,bn", TC_VARIANTS)
@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16_scaled", "tf32"])
@pytest.mark.parametrize("shape", [(7, 7, 6), (9, 8, 7), (8, 10, 8), (8, 8, 10)])
def test_single_step_tensor_core(tn, mode, shape, form, bk, bn):
    rng = np.random.default_rng(7 + sum(shape))
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], mode=mode, gemm_form=form,
                               tc_bk=bk, tc_bn=bn)
    assert kernels == ["gemm_tc"]
    check(got, ref, TOL[mode])


@pytest.mark.parametrize("mode,form,bk", [("fp16_scaled", "4m", 0), ("bf16_scaled", "4m", 0),
                                          ("tf32", "4m", 0), ("fp16_scaled", "4m", 32),
                                          ("tf32", "4m", 32), ("fp16_scaled", "3m", 0),
                                          ("tf32", "3m", 0), ("split_fp16", "auto", 0),
                                          ("split_bf16", "auto", 0), ("split_tf32", "auto", 0)])
@pytest.mark.parametrize("shape", [(13, 6, 6), (12, 6, 9), (6, 13, 7), (14, 6, 3), (13, 5, 5),
                                   (5, 14, 5), (12, 5, 8), (13, 5, 3)])
def test_narrow_results_on_the_64_and_32_column_tiles(tn, mode, form, bk, shape):
    # a result 64 or 32 wide on one side (App. A.2: n >= 32 keeps the tensor cores busy): the
    # 128 x 64 or 128 x 32 tile, the wide side taken as M whichever operand holds it; short 4M
    # contractions on the persistent kernel unless a K tile is asked for (then one tile per
    # CTA); 2 slices in flight
    rng = np.random.default_rng(900 + 3 * shape[0] + 5 * shape[1] + shape[2])
    tensors, labels, out = single_step(rng, *shape, scale=2.0 ** -8)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, [(0, 1)], (), mode=mode, gemm_form=form, tc_bk=bk,
                   sync_each_call=True)
    si = plan.step_info(0)
    narrow = min(shape[0], shape[1])
    if form == "4m" and bk == 0:   # persistent: 29-33 (64 columns), 34-38 (32 columns)
        lo, hi = (29, 33) if narrow == 6 else (34, 38)
    elif "split" in mode:          # persistent compensated: 44-48 (64), 49-53 (32 columns)
        lo, hi = (44, 48) if narrow == 6 else (49, 53)
    else:                          # one tile per CTA: 17-22 (64 columns), 23-28 (32 columns)
        lo, hi = (17, 22) if narrow == 6 else (23, 28)
    assert si["kernel_name"] == "gemm_tc" and lo <= si["tc_variant"] <= hi
    assert si["log2_m"] == max(shape[0], shape[1]) and si["log2_n"] == narrow
    check(plan.contract_host(), ref, TOL[mode])
    plan.close()
    net.close()
    # slice weights that do not cancel (a sum v0 + v1 near 0 would magnify the relative error)
    A, B = tensors
    v = np.array([1.0 + 0.25j, 0.6 - 0.3j])
    t2 = [A[None] * v.reshape(2, *([1] * A.ndim)), B, np.ones(2, complex)]
    l2 = [[900] + labels[0], labels[1], [900]]
    ref2 = O.contract(t2, l2, out, [(0, 1), (0, 2)])
    got2, info, k2 = gpu_amps(tn, t2, l2, out, [(0, 1), (0, 2)], [900], mode=mode,
                              gemm_form=form, tc_bk=bk)
    assert info["slices_in_flight"] == 2 and k2[0] == "gemm_tc"
    check(got2, ref2, TOL[mode])


@pytest.mark.parametrize("mode", ["split_fp16", "split_bf16", "split_tf32"])
@pytest.mark.parametrize("bn", [0, 256])
@pytest.mark.parametrize("shape", [(7, 7, 6), (9, 8, 7), (8, 10, 10), (10, 10, 3)])
def test_compensated_products_on_tensor_cores(tn, mode, bn, shape):
    rng = np.random.default_rng(110 + sum(shape))
    tensors, labels, out = single_step(rng, *shape, scale=2.0 ** -12)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], mode=mode, tc_bn=bn)
    assert kernels == ["gemm_tc"]
    check(got, ref, TOL[mode])


@pytest.mark.parametrize("topk", [1, 2])
def test_mixed_precision_top_k(tn, topk):
    # two dense steps: the larger runs single-pass FP16 (top-1), the smaller compensated
    rng = np.random.default_rng(140)
    a, k1, b, c = (list(range(o, o + w)) for o, w in ((0, 8), (100, 7), (200, 8), (300, 8)))
    tensors = [crandn(rng, 15, 2.0 ** -6), crandn(rng, 15, 2.0 ** -6), crandn(rng, 16)]
    labels = [a + k1, k1 + b, b + c]
    out = [int(x) for x in rng.permutation(a + c)]
    path = [(0, 1), (0, 2)]
    ref = O.contract(tensors, labels, out, path)
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, path, (), mode="mixed", mixed_topk=topk)
    forms = [plan.step_info(i)["gemm_form"] for i in range(2)]
    assert forms == ([3, 1] if topk == 1 else [1, 1])
    check(plan.contract_host(), ref, TOL["mixed"])
    plan.close()
    net.close()


def chain_of_dense_steps(rng, lks=(7, 8, 9, 10, 11)):
    # X0[a, k0] X1[k0, b1] X2[b1, b2] ...: contracted left to right, every step is a dense GEMM
    # (m = n = 2^8) with k = 2^lks[i], so T_cc grows along the path
    a = list(range(0, 8))
    bonds = [list(range(100 * (i + 1), 100 * (i + 1) + w)) for i, w in enumerate(lks)]
    outs = [list(range(1000 + 10 * i, 1000 + 10 * i + 8)) for i in range(len(lks))]
    tensors = [crandn(rng, 8 + lks[0], 2.0 ** -(lks[0] / 2))]
    labels = [a + bonds[0]]
    for i in range(len(lks)):
        nxt = bonds[i + 1] if i + 1 < len(lks) else outs[-1]
        if i + 1 < len(lks):
            tensors.append(crandn(rng, lks[i] + lks[i + 1], 2.0 ** -(lks[i + 1] / 2)))
        else:
            tensors.append(crandn(rng, lks[i] + 8))
        labels.append(bonds[i] + nxt)
    out = a + outs[-1]
    path = [(0, i) for i in range(1, len(tensors))]
    return tensors, labels, out, path


def expected_forms(plan, nd, k):
    # the k steps with the largest T_cc (ties: the earlier step first) single-pass (form 1),
    # the others compensated (form 3)
    tcc = [plan.step_info(i)["tcc"] for i in range(nd)]
    top = sorted(range(nd), key=lambda i: -tcc[i])[:k]
    return [1 if i in top else 3 for i in range(nd)]


def predicted_eps(u, single, split):
    # the error model of the precision policy (tn.h): c u per single-pass step, 4e-6 per
    # compensated step, a 1e-5 floor, in quadrature
    cu = 1.5 * np.sqrt(2 / 7) * u
    return np.sqrt(single * cu ** 2 + split * 4e-6 ** 2 + 1e-5 ** 2)


@pytest.mark.parametrize("mode,budget,u", [("bf16_scaled", 0.0, 2.0 ** -8),
                                           ("bf16_scaled", 3.5e-3, 2.0 ** -8),
                                           ("fp16_scaled", 6e-4, 2.0 ** -11),
                                           ("tf32", 6e-4, 2.0 ** -11),
                                           ("mixed", 6e-4, 2.0 ** -11)])
def test_error_budget_picks_single_pass_steps(tn, mode, budget, u):
    # Sec. 4.3 / Table 3 with an error budget: the largest-T_cc dense steps run single-pass,
    # as many as the error model allows, the rest compensated; the measured error stays
    # within the budget (BF16-scaled has a default budget of 5e-3)
    rng = np.random.default_rng(150)
    tensors, labels, out, path = chain_of_dense_steps(rng)
    ref = O.contract(tensors, labels, out, path)
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, path, (), mode=mode, eps_budget=budget)
    info = plan.info()
    nd = len(path)
    assert info["num_tc_steps"] == nd
    bud = budget if budget > 0 else 5e-3
    want = max(k for k in range(nd + 1) if k == 0 or predicted_eps(u, k, nd - k) <= bud)
    assert info["num_single_pass"] == want and info["num_compensated"] == nd - want
    assert abs(info["eps_predicted"] - predicted_eps(u, want, nd - want)) < 1e-12
    forms = [plan.step_info(i)["gemm_form"] for i in range(nd)]
    assert forms == expected_forms(plan, nd, want)
    check(plan.contract_host(), ref, bud)
    plan.close()
    net.close()


def test_mixed_topk_caps_single_pass_modes(tn):
    # mixed_topk bounds the single-pass steps of the FP16-scaled mode too
    rng = np.random.default_rng(151)
    tensors, labels, out, path = chain_of_dense_steps(rng, (7, 8, 9))
    ref = O.contract(tensors, labels, out, path)
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, path, (), mode="fp16_scaled", mixed_topk=1)
    assert [plan.step_info(i)["gemm_form"] for i in range(3)] == expected_forms(plan, 3, 1)
    assert plan.info()["num_single_pass"] == 1
    check(plan.contract_host(), ref, TOL["fp16_scaled"])
    plan.close()
    net.close()


@pytest.mark.parametrize("shape", [(10, 10, 3), (11, 9, 4), (7, 13, 5)])
def test_short_contraction_on_tensor_cores(tn, shape):
    # k = 8..32 with a large output: the K tile is zero-filled past k by the tensor map
    rng = np.random.default_rng(70 + sum(shape))
    tensors, labels, out = single_step(rng, *shape)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    for mode in ("fp16_scaled", "bf16_scaled", "tf32"):
        got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], mode=mode)
        assert kernels == ["gemm_tc"]
        check(got, ref, TOL[mode])


@pytest.mark.parametrize("mode", ["fp16_scaled", "tf32"])
@pytest.mark.parametrize("lm,ln,lk,nsl", [(12, 10, 8, 3), (7, 7, 9, 0), (9, 8, 8, 2),
                                         (12, 10, 6, 3), (10, 10, 4, 0), (11, 9, 3, 0),
                                         (14, 6, 8, 2), (13, 5, 4, 0), (6, 14, 4, 1),
                                         (15, 5, 6, 1), (13, 6, 3, 0)])
def test_persistent_short_k_kernel_over_slices(tn, mode, lm, ln, lk, nsl):
    # short contractions run on the persistent kernel (variant 12 / 13): each CTA walks tiles of
    # all slices in flight with a double-buffered accumulator; fewer tiles than SMs included
    # (nsl of the lk contracted labels are sliced, leaving k = 2^(lk - nsl))
    rng = np.random.default_rng(600 + lm + 3 * ln + 7 * lk + nsl)
    tensors, labels, out = single_step(rng, lm, ln, lk)
    K = [l for l in labels[0] if l >= 200]
    sliced = [int(x) for x in rng.choice(K, size=nsl, replace=False)] if nsl else []
    ref = O.contract(tensors, labels, out, [(0, 1)])
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, [(0, 1)], sliced, mode=mode, sync_each_call=True)
    si = plan.step_info(0)
    # rows of 16 / 32 / 64 bytes hold exactly k for k = 8 / 16 (16-bit) and k = 8 (TF32)
    k = lk - nsl
    want = {3: 16}.get(k, 13) if mode == "tf32" else {3: 14, 4: 15}.get(k, 12)
    # results 64 or 32 wide: the same kernel with 64- or 32-column tiles (variants + 17 / + 22)
    want += {6: 17, 5: 22}.get(min(lm, ln), 0)
    assert si["kernel_name"] == "gemm_tc" and si["tc_variant"] == want
    check(plan.contract_host(), ref, TOL[mode])
    plan.close()
    net.close()


def test_persistent_kernel_far_input_scales(tn):
    # inputs near 2^-70: the exponents of the operand planes sum to far below -126, so the
    # epilogue scales with two power-of-two factors instead of one (results near 2^-137, FP32
    # subnormals, still within the tolerance)
    rng = np.random.default_rng(77)
    tensors, labels, out = single_step(rng, 12, 9, 5, scale=2.0 ** -70)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], mode="fp16_scaled")
    assert kernels == ["gemm_tc"]
    check(got, ref, TOL["fp16_scaled"])


def test_checkpointed_contraction_on_the_gpu(tn, tmp_path):
    # slice chunks through the C ABI, interrupted after the first chunk and resumed
    from paper_2310_03978_gb300 import shard
    wl = W.small_workload()
    net = wl.network
    sliced = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    ref = O.contract_network(net, wl.path)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.Plan(tnet, wl.path, sliced, mode="c64", max_slices_in_flight=2)
    ck = str(tmp_path / "ck.npz")

    class Stop(Exception):
        pass

    def stop(nxt):
        if nxt == 2:
            raise Stop()

    with pytest.raises(Stop):
        shard.contract_resumable(plan, 0, 8, ck, on_chunk=stop)
    check(shard.contract_resumable(plan, 0, 8, ck), ref, TOL["c64"])
    plan.close()
    tnet.close()


def test_bounded_wait_reports_timeout_and_context_survives(tn):
    # a tensor-core CTA whose producer issues no copies: its MMA warp's wait runs out after
    # 200 ms, the kernel records the timeout and exits; the context stays usable
    status = tn.lib().tn_selftest_wait_timeout(200, None)
    assert status == 6  # TN_ERR_TIMEOUT
    wl = W.small_workload()
    net = wl.network
    got, _, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path,
                         mode="fp16_scaled")
    check(got, O.contract_network(net, wl.path), TOL["fp16_scaled"])


def test_tensor_core_scaling_keeps_tiny_magnitudes(tn):
    # amplitude-like magnitudes (2^-40) would flush to zero in FP16 without the 2^e scaling
    rng = np.random.default_rng(3)
    tensors, labels, out = single_step(rng, 8, 8, 7, scale=2.0 ** -20)
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, _, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], mode="fp16_scaled")
    assert kernels == ["gemm_tc"]
    check(got, ref, TOL["fp16_scaled"])


def test_tensor_core_step_with_slices_in_flight(tn):
    # the dense step depends on the sliced bond x; 2 slices run in one launch
    rng = np.random.default_rng(11)
    A = crandn(rng, 16)
    B = crandn(rng, 15)
    v = crandn(rng, 1)
    la = [500] + list(range(0, 8)) + list(range(200, 207))
    lb = list(range(100, 108)) + list(range(200, 207))
    out = list(rng.permutation(list(range(100, 108)) + list(range(0, 8))))
    out = [int(x) for x in out]
    tensors, labels, path = [A, B, v], [la, lb, [500]], [(0, 1), (0, 2)]
    ref = O.contract(tensors, labels, out, path)
    for mode in ("c64", "fp16_scaled"):
        got, info, kernels = gpu_amps(tn, tensors, labels, out, path, [500], mode=mode)
        assert info["slices_in_flight"] == 2
        assert kernels[0] == ("gemm_tc" if mode == "fp16_scaled" else "gemm_simt")
        check(got, ref, TOL[mode])


@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
@pytest.mark.parametrize("lm,ln,lk,nsl", [(10, 4, 8, 3), (14, 3, 8, 0), (6, 9, 12, 2)])
def test_large_leaves_tiled_permutation_with_slices(tn, mode, lm, ln, lk, nsl):
    # leaves of rank >= 12 are bound by the tiled permutation kernel: random label orders, and
    # sliced labels (contracted between A and B) at random source bit positions
    rng = np.random.default_rng(300 + lm + 7 * ln + 13 * lk + nsl)
    tensors, labels, out = single_step(rng, lm, ln, lk)
    K = [l for l in labels[0] if l >= 200]
    sliced = [int(x) for x in rng.choice(K, size=nsl, replace=False)] if nsl else []
    ref = O.contract(tensors, labels, out, [(0, 1)])
    got, info, kernels = gpu_amps(tn, tensors, labels, out, [(0, 1)], sliced, mode=mode)
    assert info["num_slices"] == 1 << nsl
    check(got, ref, TOL[mode])


@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
def test_graph_replay_matches_direct_launches(tn, mode):
    wl = W.small_workload()
    net = wl.network
    sl = W.greedy_slices(net.labels, net.open_labels, wl.path, 2)
    tnet = tn.Network.from_workload(net)
    direct = tn.Plan(tnet, wl.path, sl, mode=mode)
    graph = tn.Plan(tnet, wl.path, sl, mode=mode, use_graph=True, max_slices_in_flight=2)
    ref = direct.contract_host()
    for _ in range(3):  # capture on first use, then replays
        got = graph.contract_host()
        check(got, ref, 1e-6)
    part = graph.contract_host(1, 4)   # a partial batch runs without the graph
    check(part, O.contract_network(net, wl.path, sl, 1, 4), TOL[mode])
    direct.close()
    graph.close()
    tnet.close()


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16_scaled", "split_fp16", "split_bf16",
                                  "tf32", "split_tf32"])
@pytest.mark.parametrize("lk1,first", [(7, "gemm_tc"), (5, "gemm_simt"), (1, "generic")])
def test_chained_steps_feed_the_tensor_cores(tn, lk1, first, mode):
    # step 1 writes the operand of tensor-core step 2 directly as planar 16-bit numbers, with an
    # exponent bounded from its own inputs' max-abs (the tensor-core and CUDA-core epilogues)
    rng = np.random.default_rng(40 + lk1)
    a, k1, b, c = (list(range(o, o + w)) for o, w in ((0, 8), (100, lk1), (200, 8), (300, 8)))
    T0 = crandn(rng, 8 + lk1, 2.0 ** -6)
    T1 = crandn(rng, lk1 + 8, 2.0 ** -6)
    T2 = crandn(rng, 16, 2.0 ** -4)
    tensors, labels = [T0, T1, T2], [a + k1, k1 + b, b + c]
    out = [int(x) for x in rng.permutation(a + c)]
    path = [(0, 1), (0, 2)]
    ref = O.contract(tensors, labels, out, path)
    for form in (("4m", "3m") if "split" not in mode else ("auto",)):
        got, _, kernels = gpu_amps(tn, tensors, labels, out, path, mode=mode, gemm_form=form)
        assert kernels == [first, "gemm_tc"]
        check(got, ref, TOL[mode])


@pytest.mark.parametrize("mode", ["fp16_scaled", "bf16_scaled", "split_fp16", "tf32"])
@pytest.mark.parametrize("nsl", [0, 1])
@pytest.mark.parametrize("thin_tc", [1, -1])
def test_thin_step_feeds_the_tensor_cores(tn, mode, nsl, thin_tc):
    # step 1 is thin (2^11 x 8, k = 4: the streaming kernel) and its result is an operand of
    # the tensor-core step 2 (m = 2^7, n = 2^8, k = 2^7): for single-pass consumers it writes
    # the planar 16-bit copy itself, with an exponent bounded from its inputs' max-abs (its
    # inputs are leaves, measured by an amax pass; at these magnitudes, ~2^-60 after step 1, an
    # unscaled FP16 copy would flush to zero)
    rng = np.random.default_rng(45 + nsl)
    a = list(range(0, 11))
    k1 = [100, 101]
    b = [200, 201, 202]
    c = list(range(300, 308))
    tensors = [crandn(rng, 13, 2.0 ** -30), crandn(rng, 5, 2.0 ** -30),
               crandn(rng, 15, 2.0 ** -6)]
    labels = [a + k1, k1 + b, a[7:] + b + c]
    out = [int(x) for x in rng.permutation(a[:7] + c)]
    path = [(0, 1), (0, 2)]
    sliced = [a[9]] if nsl else []
    ref = O.contract(tensors, labels, out, path)
    got, info, kernels = gpu_amps(tn, tensors, labels, out, path, sliced, mode=mode,
                                  thin_tc=thin_tc)
    first = "thin_tc" if thin_tc > 0 else "stream"
    assert kernels == [first, "gemm_tc"]
    check(got, ref, TOL[mode])


@pytest.mark.parametrize("form", ["auto", "4m", "3m"])
def test_autotuned_plan_matches_oracle(tn, form):
    # the first full batch times every applicable tensor-core variant per step; results before
    # and after tuning agree with the oracle
    rng = np.random.default_rng(90)
    a, k1, b, c = (list(range(o, o + w)) for o, w in ((0, 9), (100, 7), (200, 8), (300, 8)))
    tensors = [crandn(rng, 16, 2.0 ** -6), crandn(rng, 15, 2.0 ** -6), crandn(rng, 16)]
    labels = [a + k1, k1 + b, b + c]
    out = [int(x) for x in rng.permutation(a + c)]
    path = [(0, 1), (0, 2)]
    ref = O.contract(tensors, labels, out, path)
    net = tn.Network(tensors, labels, out)
    plan = tn.Plan(net, path, (), mode="fp16_scaled", gemm_form=form, autotune=True)
    for _ in range(3):
        check(plan.contract_host(), ref, TOL["fp16_scaled"])
    variants = [plan.step_info(i)["tc_variant"] for i in range(2)]
    assert all(v >= 0 for v in variants)
    forms = [plan.step_info(i)["gemm_form"] for i in range(2)]
    if form == "4m":
        assert forms == [1, 1]
    if form == "3m":
        assert forms == [2, 2]
    plan.close()
    net.close()


def test_host_entry_points_and_set_data(tn):
    wl = W.small_workload()
    net = wl.network
    tnet = tn.Network.from_workload(net)
    plan = tn.Plan(tnet, wl.path, (), mode="c64")
    got = plan.contract_host()
    check(got, O.contract_network(net, wl.path), 1e-5)
    # new numbers, same structure: conjugated tensors give the conjugate circuit
    tnet.set_data([np.conj(t) for t in net.tensors])
    got2 = plan.contract_host()
    check(got2, np.conj(O.contract_network(net, wl.path)), 1e-5)
    with pytest.raises(tn.TnError):
        plan.contract_host(0, 2)  # one slice only
    plan.close()
    tnet.close()


def test_caller_workspace_is_used_and_misalignment_rejected(tn):
    wl = W.small_workload()
    net = wl.network
    tnet = tn.Network.from_workload(net)
    ws = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    plan = tn.Plan(tnet, wl.path, (), mode="c64", workspace=ws)
    assert plan.info()["workspace_bytes"] <= ws.numel()
    check(plan.contract_host(), O.contract_network(net, wl.path), 1e-5)
    plan.close()
    with pytest.raises(tn.TnError) as e:
        tn.Plan(tnet, wl.path, (), mode="c64", workspace=ws[8:])  # 8 bytes past 256 alignment
    assert e.value.status == 1  # TN_ERR_INVALID_ARG
    tnet.close()


# ------------------------------------------------------------------ the full-size circuit
@pytest.mark.parametrize("mode,form", [("c64", "auto"), ("fp16_scaled", "4m"),
                                       ("fp16_scaled", "3m"), ("split_fp16", "auto"),
                                       ("mixed", "auto"), ("bf16_scaled", "4m"),
                                       ("tf32", "auto"), ("split_tf32", "auto")])
def test_bench_circuit_full_size(tn, mode, form):
    golden = os.path.join(HERE, "golden", "sycamore_5x6_c14_open10_s4.amps.txt")
    if not os.path.exists(golden):
        pytest.skip("golden amplitudes not generated")
    wl = W.bench_workload()
    net = wl.network
    ref = read_golden("sycamore_5x6_c14_open10_s4")
    got, info, kernels = gpu_amps(tn, net.tensors, net.labels, net.open_labels, wl.path,
                                  wl.sliced, mode=mode, gemm_form=form,
                                  autotune=mode != "c64")
    assert info["num_slices"] == 16 and info["max_log2_size"] <= 28
    check(got, ref, CIRCUIT_TOL[mode])
    n = wl.circuit.n_qubits
    x_ref = O.readout(ref, n)[3]
    x_got = O.readout(got, n)[3]
    assert abs(x_got - x_ref) / abs(x_ref) <= 1e-3
    if mode == "fp16_scaled":
        assert "gemm_tc" in kernels
    if mode == "bf16_scaled":
        # the policy's prediction holds the bar and the largest step stays single-pass
        assert info["num_single_pass"] >= 1
        assert info["eps_predicted"] <= TOL[mode]


# ------------------------------------------------------------------ optimised paths (Sec. 3.2)
@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
def test_annealed_path_with_dynamic_slices(tn, mode):
    # the small circuit along a path and slices from the annealing optimiser
    wl = W.small_workload()
    net = wl.network
    ref = read_golden("sycamore_3x4_c8_open6")
    path, sliced, info = tn.path_optimize(net.labels, net.open_labels, wl.path, seed=11,
                                          sweeps=100, sweeps_per_slice=20, sweeps_final=50,
                                          t_start=0.1, t_end=0.001, max_log2_size=7)
    assert info["num_sliced"] >= 1
    got, pinfo, _ = gpu_amps(tn, net.tensors, net.labels, net.open_labels, path, sliced,
                             mode=mode)
    assert pinfo["max_log2_size"] <= 7
    check(got, ref, TOL[mode])


def test_bench_circuit_on_an_annealed_path(tn):
    golden = os.path.join(HERE, "golden", "sycamore_5x6_c14_open10_s4.amps.txt")
    if not os.path.exists(golden):
        pytest.skip("golden amplitudes not generated")
    wl = W.bench_workload()
    net = wl.network
    ref = read_golden("sycamore_5x6_c14_open10_s4")
    path, sliced, info = tn.path_optimize(net.labels, net.open_labels, wl.path, seed=7,
                                          sweeps=300, sweeps_per_slice=40, sweeps_final=200,
                                          t_start=0.03, t_end=0.001, max_log2_size=28, chains=8)
    assert info["max_log2_size"] <= 28
    got, pinfo, kernels = gpu_amps(tn, net.tensors, net.labels, net.open_labels, path, sliced,
                                   mode="fp16_scaled")
    check(got, ref, CIRCUIT_TOL["fp16_scaled"])
    n = wl.circuit.n_qubits
    x_ref, x_got = O.readout(ref, n)[3], O.readout(got, n)[3]
    assert abs(x_got - x_ref) / abs(x_ref) <= 1e-3


# ------------------------------------------------------------------ amplitude batches (a10)
@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
def test_sliced_open_labels_give_amplitude_batches(tn, mode):
    # two of the six open labels sliced along with three bonds: 32 slices, each added into the
    # amplitude block its open bits select; whole range, split ranges and graph replay all give
    # the oracle's (unsliced) amplitudes
    wl = W.small_workload()
    net = wl.network
    ref = O.contract_network(net, wl.path)
    bonds = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    sliced = bonds + [net.open_labels[4], net.open_labels[1]]  # slice bits 3, 4: open bits
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.Plan(tnet, wl.path, sliced, mode=mode, sync_each_call=True,
                   max_slices_in_flight=6)
    info = plan.info()
    assert info["num_open_sliced"] == 2 and info["num_slices"] == 32
    check(plan.contract_host(), ref, TOL[mode])
    split = plan.contract_host(0, 13) + plan.contract_host(13, 32)
    check(split, ref, TOL[mode])
    # slices 0..7 have 0 for both sliced open labels (amplitude bits 1 and 4): only that block
    # of the amplitudes is set
    part = plan.contract_host(0, 8)
    idx = np.arange(64)
    in_block = ((idx >> (5 - 4)) & 1) == 0
    in_block &= ((idx >> (5 - 1)) & 1) == 0
    assert np.all(part[~in_block] == 0)
    plan.close()
    graph = tn.Plan(tnet, wl.path, sliced, mode=mode, use_graph=True, max_slices_in_flight=8)
    for _ in range(2):
        check(graph.contract_host(), ref, TOL[mode])
    graph.close()
    tnet.close()


def test_all_open_circuit_in_64_amplitude_batches(tn):
    # every qubit of a 12-qubit circuit open, six of them sliced: 64 batches of 64 amplitudes in
    # one call, against the state vector
    circ = W.random_circuit(3, 4, 8, seed=21)
    net = W.build_network(circ, list(range(12)), {})
    path = W.greedy_path(net.labels, net.open_labels)
    sv = O.statevector(12, circ.gates)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.Plan(tnet, path, net.open_labels[:6], mode="c64", use_graph=True)
    assert plan.info()["num_slices"] == 64 and plan.info()["slices_in_flight"] == 64
    for _ in range(2):
        check(plan.contract_host(), sv, TOL["c64"])
    plan.close()
    tnet.close()


# ------------------------------------------------------------------ batched small steps (a10)
@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
def test_chained_small_steps_match_single_launches(tn, mode):
    # runs of small element-wise steps go out as one launch (one block per slice); profile mode
    # launches every step on its own: both must give the oracle's amplitudes
    wl = W.small_workload()
    net = wl.network
    sl = W.greedy_slices(net.labels, net.open_labels, wl.path, 3)
    ref = O.contract_network(net, wl.path)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    res, launches = {}, {}
    for prof in (False, True):
        plan = tn.Plan(tnet, wl.path, sl, mode=mode, profile=prof, sync_each_call=True)
        amps = torch.zeros(1 << len(net.open_labels), dtype=torch.complex128, device="cuda")
        l0 = plan.info()["kernel_launches"]
        plan.contract(amps)
        launches[prof] = plan.info()["kernel_launches"] - l0
        res[prof] = amps.cpu().numpy()
        plan.close()
    tnet.close()
    assert launches[False] < launches[True] // 4
    check(res[False], ref, TOL[mode])
    check(res[True], ref, TOL[mode])


# ------------------------------------------------------------------ sparse-state (Sec. 3.3)
def sparse_amps(tn, tensors, labels, open_labels, path, samples):
    net = tn.Network(tensors, labels, open_labels)
    plan = tn.SparsePlan(net, path, samples)
    amps = torch.zeros(len(samples), dtype=torch.complex128, device="cuda")
    plan.contract(amps)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    net.close()
    return amps.cpu().numpy(), info


def sv_index(bits):
    return int("".join(str(int(b)) for b in bits), 2)


def test_sparse_state_matches_oracle_and_state_vector(tn):
    circ = W.random_circuit(3, 4, 8, seed=31)
    net = W.build_network(circ, list(range(12)), {})
    path = W.greedy_path(net.labels, net.open_labels)
    rng = np.random.default_rng(5)
    smp = rng.integers(0, 2, size=(200, 12))
    smp[1] = smp[0]
    smp[-1] = smp[7]
    got, info = sparse_amps(tn, net.tensors, net.labels, net.open_labels, path, smp)
    ref = O.contract_sparse(net.tensors, net.labels, net.open_labels, path, smp)
    check(got, ref, TOL["c64"])
    sv = O.statevector(12, circ.gates)
    check(got, sv[[sv_index(r) for r in smp]], TOL["c64"])
    assert got[0] == got[1] and got[7] == got[-1]
    assert info["distinct_samples"] == len({tuple(r) for r in smp})
    assert info["num_steps"] == net.num_tensors - 1
    assert info["kernel_launches"] == info["num_steps"] + 2


def test_sparse_state_with_closed_qubits_and_closed_forms(tn):
    wl = W.small_workload()
    net = wl.network
    rng = np.random.default_rng(13)
    smp = rng.integers(0, 2, size=(40, len(net.open_labels)))
    got, _ = sparse_amps(tn, net.tensors, net.labels, net.open_labels, wl.path, smp)
    dense = O.contract_network(net, wl.path)
    check(got, dense[[sv_index(r) for r in smp]], TOL["c64"])
    n = 8
    g = W.build_network(W.ghz_circuit(n), list(range(n)), {})
    smp = np.array([[0] * n, [1] * n, [1] + [0] * (n - 1), [1] * n])
    got, info = sparse_amps(tn, g.tensors, g.labels, g.open_labels,
                            W.greedy_path(g.labels, g.open_labels), smp)
    np.testing.assert_allclose(got, [2 ** -0.5, 2 ** -0.5, 0, 2 ** -0.5], atol=1e-6)
    assert info["distinct_samples"] == 3


def test_sparse_state_rejects_bad_input(tn):
    circ = W.random_circuit(2, 2, 4, seed=3)
    net = W.build_network(circ, list(range(4)), {})
    path = W.greedy_path(net.labels, net.open_labels)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    with pytest.raises(tn.TnError) as e:
        tn.SparsePlan(tnet, path, np.array([[0, 1, 2, 0]]))
    assert e.value.status == 1  # TN_ERR_INVALID_ARG
    bad = list(path)
    bad[-1] = (bad[-1][0], bad[0][1])  # a retired id
    with pytest.raises(tn.TnError) as e:
        tn.SparsePlan(tnet, bad, np.zeros((3, 4)))
    assert e.value.status == 3  # TN_ERR_PATH
    tnet.close()


def test_sparse_state_tiled_steps_over_many_configurations(tn):
    # an 18-qubit all-open circuit: its larger steps run as tiled GEMMs per configuration
    circ, net, smp = W.sparse_state_workload(3, 6, 10, 512, config_id=11)
    path = W.greedy_path(net.labels, net.open_labels)
    got, info = sparse_amps(tn, net.tensors, net.labels, net.open_labels, path, smp)
    assert info["gemm_steps"] + info["grouped_steps"] > 0
    sv = O.statevector(circ.n_qubits, circ.gates)
    check(got, sv[[sv_index(r) for r in smp]], TOL["c64"])


@pytest.mark.parametrize("mode", ["c64", "fp16_scaled"])
def test_sparse_state_dense_subtrees_on_ordinary_plans(tn, mode):
    # the 24-qubit all-open circuit: the subtrees below the open bonds run as ordinary plans
    # (tensor cores in FP16-scaled mode), the rest as sparse steps
    circ, net, smp = W.sparse_state_workload(num_samples=512)
    path, _, _ = tn.path_optimize(net.labels, net.open_labels,
                                  W.greedy_path(net.labels, net.open_labels), seed=7,
                                  sweeps=500, sweeps_final=0, t_start=0.03, t_end=0.001, chains=8)
    tnet = tn.Network(net.tensors, net.labels, net.open_labels)
    plan = tn.SparsePlan(tnet, path, smp, mode=mode)
    amps = torch.zeros(len(smp), dtype=torch.complex128, device="cuda")
    plan.contract(amps)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    tnet.close()
    assert info["dense_subtrees"] > 0 and info["dense_subtree_steps"] > 0
    assert info["grouped_steps"] > 0
    sv = O.statevector(circ.n_qubits, circ.gates)
    check(amps.cpu().numpy(), sv[[sv_index(r) for r in smp]], TOL[mode])
