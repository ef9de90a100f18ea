"""tn_readout_noalloc, the allocation-free FP64 readout, against the plan-based tn_readout.

The entry point serves callers that cannot allocate device memory (their GPU memory is held by
another allocator or a fixed budget); its scratch is a fixed device array inside libtn.so.  This
file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_03978_gb300 import tn as T
    T.lib()
    return T


def test_noalloc_readout_matches_plan_readout_on_a_circuit(tn):
    from paper_2310_03978_gb300 import workload as W
    wl = W.small_workload()
    net = tn.Network.from_workload(wl.network)
    plan = tn.Plan(net, wl.path, wl.sliced, mode="c64")
    amps = torch.zeros(1 << len(wl.network.open_labels), dtype=torch.complex128, device="cuda")
    plan.contract(amps)
    ref = plan.readout(amps, wl.circuit.n_qubits)
    for _ in range(2):  # two calls in a row share the scratch array
        got = tn.readout_noalloc(amps, wl.circuit.n_qubits)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    plan.close()
    net.close()


def test_noalloc_readout_spans_many_blocks(tn):
    # 2^20 amplitudes: 16 block sums; the plan-based readout of a one-tensor network with 20
    # open labels reads the same vector
    n = 20
    g = torch.Generator(device="cuda").manual_seed(5)
    amps = torch.randn(1 << n, dtype=torch.complex128, device="cuda", generator=g) * 2.0 ** -10
    one = np.zeros((2,) * n, dtype=np.complex128)
    net = tn.Network([one], [list(range(n))], list(range(n)))
    plan = tn.Plan(net, [], (), mode="c64")
    ref = plan.readout(amps, 30)
    for _ in range(2):
        got = tn.readout_noalloc(amps, 30)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    plan.close()
    net.close()


def test_noalloc_readout_rejects_vectors_beyond_its_scratch(tn):
    amps = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = np.zeros(4)
    import ctypes as C
    status = tn.lib().tn_readout_noalloc(C.c_void_p(amps.data_ptr()), (1 << 28) + 1, 30,
                                         C.c_void_p(out.ctypes.data), None)
    assert status == 1  # TN_ERR_INVALID_ARG, before any device work
