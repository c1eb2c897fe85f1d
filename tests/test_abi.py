"""The C-ABI library: builds, loads, exports what include/qldpc.h declares, validates on the host.

No test here launches a kernel; every call below is rejected by host-side validation before any
CUDA work, or needs no device.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qldpc.h")


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    return qldpc


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"QLDPC_API\s+[\w\s\*]+?\b(qldpc_\w+)\s*\(", text)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("qldpc_graph_create", "qldpc_graph_create_csc", "qldpc_graph_destroy",
                     "qldpc_decode", "qldpc_decode_ex", "qldpc_decode_pair", "qldpc_decode_host",
                     "qldpc_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(q):
    lib = ctypes.CDLL(q.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", q.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(declared_functions()) <= exported
    # nothing else with external linkage leaks out of the library's own namespace
    assert not [s for s in exported if "qldpc" in s and not s.startswith("qldpc_")]


def test_binding_names_match_header(q):
    for name in declared_functions():
        assert callable(getattr(q, name))


def test_noalloc_scratch_size_matches_header(q):
    text = open(HEADER).read()
    m = re.search(r"QLDPC_NOALLOC_SCRATCH_BYTES\s*=\s*([0-9 *]+)", text)
    assert m
    size = 1
    for f in m.group(1).split("*"):
        size *= int(f)
    assert q.qldpc_noalloc_scratch_bytes() == size == q.QLDPC_NOALLOC_SCRATCH_BYTES


def test_status_strings(q):
    assert q.qldpc_status_string(0) == b"QLDPC_OK"
    for code in (-1, -2, -3, -4, -5):
        assert q.qldpc_status_string(code).startswith(b"QLDPC_ERR_")
    assert q.qldpc_status_string(42) == b"unknown qldpc status"


def _create(q, row_ptr, col_idx, m, n, csc=False):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    fn = q.qldpc_graph_create_csc if csc else q.qldpc_graph_create
    rc = fn(rp.ctypes.data, ci.ctypes.data if ci.size else None, m, n, ctypes.byref(h))
    if rc == 0:
        q.qldpc_graph_destroy(h)
    return rc


@pytest.mark.parametrize("row_ptr,col_idx,m,n", [
    ([0, 2], [0, 1], 0, 2),            # m <= 0
    ([0, 2], [0, 1], 1, 0),            # n <= 0
    ([1, 3], [0, 1], 1, 2),            # row_ptr[0] != 0
    ([0, 2, 1], [0, 1], 2, 2),         # decreasing row_ptr
    ([0, 2], [0, 2], 1, 2),            # column out of range
    ([0, 2], [0, -1], 1, 2),           # negative column
    ([0, 3], [0, 1, 1], 1, 2),         # repeated column in a row
    ([0, 1], [0], 1, 2),               # row degree 1
    ([0, 0, 2], [0, 1], 2, 2),         # row degree 0
])
def test_graph_create_rejects_malformed_csr(q, row_ptr, col_idx, m, n):
    assert _create(q, row_ptr, col_idx, m, n) == q.QLDPC_ERR_INVALID_ARG


def test_graph_create_rejects_null_arguments(q):
    rp = np.array([0, 2], dtype=np.int32)
    assert q.qldpc_graph_create(rp.ctypes.data, None, 1, 2, None) == q.QLDPC_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert q.qldpc_graph_create(None, None, 1, 2, ctypes.byref(h)) == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_graph_create(rp.ctypes.data, None, 1, 2, ctypes.byref(h)) == q.QLDPC_ERR_INVALID_ARG


def test_graph_create_rejects_oversized_degrees(q):
    d = q.QLDPC_MAX_ROW_DEGREE + 1
    assert _create(q, [0, d], np.arange(d), 1, d) == q.QLDPC_ERR_UNSUPPORTED
    k = q.QLDPC_MAX_COL_DEGREE + 1           # column 0 in k rows of degree 2
    rp = np.arange(0, 2 * k + 1, 2)
    ci = np.stack([np.zeros(k, int), np.arange(1, k + 1)], axis=1).ravel()
    assert _create(q, rp, ci, k, k + 1) == q.QLDPC_ERR_UNSUPPORTED


def test_graph_create_csc_validation(q):
    assert _create(q, [0, 1, 3], [0, 0, 1], 0, 2, csc=True) == q.QLDPC_ERR_INVALID_ARG
    assert _create(q, [0, 1, 3], [0, 0, 5], 2, 2, csc=True) == q.QLDPC_ERR_INVALID_ARG
    # a CSC whose rows end up with degree 1 is rejected by the CSR validation it feeds
    assert _create(q, [0, 1, 2], [0, 1], 2, 2, csc=True) == q.QLDPC_ERR_INVALID_ARG


def test_decode_rejects_null_graph(q):
    assert q.qldpc_decode(None, None, 0, None, 10, 0.75, None, None, None) == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_decode_ex(None, None, 0, None, 10, 0.75, None, None, None, None, 0, 0, None) \
        == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_decode_host(None, None, 0, None, 10, 0.75, None, None, None, 0, 0, None) \
        == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_graph_dims(None, None, None, None, None, None) == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_graph_footprint(None, 0, None, None) == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_graph_set_launch(None, 0, 0, 0) == q.QLDPC_ERR_INVALID_ARG
    q.qldpc_graph_destroy(None)


def test_learned_entry_points_validate_on_the_host(q):
    inv = q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_graph_set_weights(None, None, 0) == inv
    size = ctypes.c_size_t()
    assert q.qldpc_nms_workspace_bytes(None, 16, 4, ctypes.byref(size)) == inv
    assert q.qldpc_nms_forward(None, None, None, 16, None, None, 4, None, 0, None, None, None, 0, None) == inv
    assert q.qldpc_nms_backward(None, None, None, 16, None, 4, None, 0, None, None, None, 0, None) == inv
    # an unknown loss kind is refused before anything else is looked at
    assert q.qldpc_nms_forward(None, None, None, 16, None, None, 4, None, 7, None, None, None, 0, None) == inv
    assert q.qldpc_nms_backward(None, None, None, 16, None, 4, None, -1, None, None, None, 0, None) == inv
    assert q.qldpc_adam_step(None, None, None, None, -1, 1, 1e-3, 0.9, 0.999, 1e-8, None) == inv
    assert q.qldpc_adam_step(None, None, None, None, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None) == inv
    assert q.qldpc_adam_step(None, None, None, None, 10, 1, 1e-3, 1.0, 0.999, 1e-8, None) == inv
    assert q.qldpc_adam_step(None, None, None, None, 0, 1, 1e-3, 0.9, 0.999, 1e-8, None) == q.QLDPC_OK
    assert q.qldpc_sample_errors(None, 1, 0, 4, 0.01, 0.02, None, None, None) == inv
    assert q.qldpc_logical_failures(None, 0, 10, None, None, None, 4, None, None) == inv
    assert q.qldpc_logical_failures(None, 2, 10, None, None, None, 0, None, None) == q.QLDPC_OK
    assert q.qldpc_logical_failures(None, 2, 10, None, None, None, 4, None, None) == inv
    # (k + 1) words of ceil(n/32) must fit in 48 KB of shared memory
    assert q.qldpc_logical_failures(ctypes.c_void_p(16), 400, 1000, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                    ctypes.c_void_p(16), 4, ctypes.c_void_p(16), None) == q.QLDPC_ERR_UNSUPPORTED


def test_product_and_oracle_are_independent():
    """The decoder package never touches the oracle, and the oracle imports nothing of the package."""
    pkg = os.path.join(ROOT, "paper_2508_07879_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "qldpc_oracle" not in text and "liboracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2508_07879_gb300" not in text, f
            assert "qldpc.h" not in text and "msa_kernel" not in text, f


def test_binding_refuses_host_tensors(q):
    """No CPU fallback: device arguments given as host tensors are refused before the library is
    called, for the decode and the soft-syndrome decode alike."""
    import torch

    class FakeGraph:            # only the dimensions are read before the arguments are marshalled
        m, n, handle = 4, 6, ctypes.c_void_p(0)

    syn = torch.zeros((2, 4), dtype=torch.uint8)
    prior = torch.ones(6)
    with pytest.raises(TypeError, match="CUDA tensor"):
        q.decode(FakeGraph(), syn, prior, 10)
    soft = FakeGraph()
    soft.n = 10                 # [H | I_4] of a 4 x 6 H
    with pytest.raises(TypeError, match="CUDA tensor"):
        q.decode_soft(soft, syn, prior, torch.ones(4), 10)
    with pytest.raises(ValueError, match="data-syndrome"):
        q.decode_soft(soft, syn, torch.ones(5), torch.ones(4), 10)
