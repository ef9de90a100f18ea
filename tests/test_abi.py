"""The C ABI library loads, exports every symbol that include/tn.h declares, and rejects bad
input on the host before any device work (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from paper_2310_03978_gb300 import tn as T
from paper_2310_03978_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tn.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return T.lib()


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(T.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(9):
        assert lib.tn_status_string(code)
    assert lib.tn_status_string(0) == b"ok"


def _load(tensors, labels, open_labels):
    return T.Network(tensors, labels, open_labels)


def test_rejects_dim_other_than_two(lib):
    with pytest.raises(T.TnError) as e:
        _load([np.ones(3, complex), np.ones(3, complex)], [[0], [0]], [])
    assert e.value.status == 7  # TN_ERR_UNSUPPORTED


def test_rejects_dangling_label(lib):
    with pytest.raises(T.TnError) as e:
        _load([np.ones((2, 2), complex), np.ones(2, complex)], [[0, 1], [0]], [])
    assert e.value.status == 2  # TN_ERR_SHAPE


def test_rejects_repeated_and_unknown_open_labels(lib):
    with pytest.raises(T.TnError) as e:
        _load([np.ones((2, 2), complex)], [[0, 1]], [0, 0])
    assert e.value.status == 2
    with pytest.raises(T.TnError) as e:
        _load([np.ones((2, 2), complex)], [[0, 1]], [0, 5])
    assert e.value.status == 2


def test_rejects_label_out_of_range(lib):
    with pytest.raises(T.TnError) as e:
        _load([np.ones(2, complex), np.ones(2, complex)], [[-1], [-1]], [])
    assert e.value.status == 1


def test_error_detail_is_readable(lib):
    with pytest.raises(T.TnError) as e:
        _load([np.ones(3, complex), np.ones(3, complex)], [[0], [0]], [])
    assert "dim" in e.value.detail


def test_workload_networks_pass_host_validation_shape_rules():
    # the generator's networks obey the loader's label rule (2 holders, or 1 + open)
    for wl in (W.small_workload(),):
        cnt = {}
        for ls in wl.network.labels:
            for l in ls:
                cnt[l] = cnt.get(l, 0) + 1
        for l in wl.network.open_labels:
            cnt[l] += 1
        assert all(v == 2 for v in cnt.values())
