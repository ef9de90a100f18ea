"""The binding refuses amplitude buffers a kernel would overrun, before any call into libtn.so.

Each kernel behind tn_contract, tn_readout, tn_readout_noalloc and tn_sparse_contract reads or
writes a fixed number of complex128 values at the address it is given; a tensor of another
dtype, size or stride, or one in host memory, must be rejected in Python.  These checks run
without a GPU (the host tensors are rejected on their dtype, layout or size first, and on
their device last).
"""
import pytest

torch = pytest.importorskip("torch")

from paper_2310_03978_gb300 import tn as T  # noqa: E402


class _Net:
    num_open = 4


def _plan():
    p = T.Plan.__new__(T.Plan)
    p.network = _Net()
    p.handle = None
    return p


def _sparse():
    p = T.SparsePlan.__new__(T.SparsePlan)
    p.num_samples = 16
    p.handle = None
    return p


BAD = [
    (torch.zeros(16, dtype=torch.complex64), TypeError, "complex128"),
    (torch.zeros(16, dtype=torch.float64), TypeError, "complex128"),
    (torch.zeros(32, dtype=torch.complex128)[::2], ValueError, "contiguous"),
    (torch.zeros(8, dtype=torch.complex128), ValueError, "16 entries"),
    (torch.zeros(16, dtype=torch.complex128), ValueError, "CUDA"),
]


@pytest.mark.parametrize("amps,exc,msg", BAD)
def test_plan_calls_reject_bad_amplitude_buffers(amps, exc, msg):
    with pytest.raises(exc, match=msg):
        _plan().contract(amps, 0, 1)
    with pytest.raises(exc, match=msg):
        _plan().readout(amps, 4)
    with pytest.raises(exc, match=msg):
        _sparse().contract(amps)


@pytest.mark.parametrize("amps,exc,msg", [b for b in BAD if "entries" not in b[2]] +
                         [(torch.zeros(0, dtype=torch.complex128), ValueError, "empty")])
def test_noalloc_readout_rejects_bad_buffers(amps, exc, msg):
    with pytest.raises(exc, match=msg):
        T.readout_noalloc(amps, 4)


def test_contract_host_rejects_bad_output_arrays():
    import numpy as np
    p = _plan()
    for out in (np.zeros(16, np.complex64), np.zeros(8, np.complex128),
                np.zeros(32, np.complex128)[::2]):
        with pytest.raises(ValueError):
            p.contract_host(0, 1, out=out)


def test_network_rejects_label_counts_that_do_not_match_ranks():
    # one label per axis, rank-0 tensors included (no labels); checked before libtn.so is called
    import numpy as np
    with pytest.raises(ValueError, match="one label per axis"):
        T.Network([np.ones((2, 2), complex)], [[0]], [0])
    with pytest.raises(ValueError, match="one label per axis"):
        T.Network([np.complex128(1.0)], [[0]], [])
    with pytest.raises(ValueError, match="one label per axis"):
        T.Network([np.ones(2, complex), np.ones(2, complex)], [[0]], [])
