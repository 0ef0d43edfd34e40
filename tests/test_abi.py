"""The C-ABI library loads, exports every entry point of include/tmotif.h and
rejects malformed input before touching the device (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tmotif.h")


@pytest.fixture(scope="module")
def tm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2001_07158_gb300 as tm

    return tm


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tmotif_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tmotif_create_graph", "tmotif_destroy_graph", "tmotif_decide", "tmotif_extract",
                     "tmotif_submit", "tmotif_poll", "tmotif_server_create", "tmotif_server_destroy",
                     "tmotif_last_error", "tmotif_decide_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(tm):
    lib = C.CDLL(tm.LIB_PATH)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_names_match_the_abi(tm):
    for f in declared_functions():
        assert hasattr(tm, f), f


def _desc_args(n=4):
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 3], np.uint32)
    time = np.array([1, 2, 3], np.uint32)
    color = np.zeros(n, np.uint32)
    return n, src, dst, time, color


def test_invalid_descriptors_are_rejected_without_a_device(tm):
    # checks that need no device: no colours, missing arrays (edge ids, times
    # and colours are validated on the device; see tests/test_gpu_parity.py)
    n, src, dst, time, color = _desc_args()
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_create_graph(n, src, dst, time, color, 0)
    assert e.value.code == 1
    lib = C.CDLL(tm.LIB_PATH)
    lib.tmotif_create_graph.argtypes = [C.c_void_p, C.c_void_p]
    h = C.c_void_p()
    assert lib.tmotif_create_graph(None, C.byref(h)) == 1
    assert lib.tmotif_create_graph(C.c_void_p(0), None) == 1


def test_last_error_is_never_null(tm):
    assert isinstance(tm.tmotif_last_error(), str)
