"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point include/qtp.h declares; host-side argument validation rejects bad
calls before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtp.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"QTP_API\s+[\w\s\*]+?\b(qtp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_14318_gb300 import build, qtp
    build.build()
    return qtp.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("qtp_plan_create", "qtp_forward", "qtp_backward", "qtp_forward_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2212_14318_gb300 import qtp
    for name in declared_functions():
        assert hasattr(lib, name), f"libqtp does not export {name}"
        assert name in qtp.SIGNATURES, f"binding has no signature for {name}"


def test_version(lib):
    assert lib.qtp_version() >= 100


@pytest.mark.parametrize("dims,status", [((0, 4, 4, 4), 1), ((4, -1, 4, 4), 1), ((4, 4, 0, 4), 1),
                                         ((4, 4, 4, 0), 1), ((4, 4, 4, 5000), 2),
                                         ((1 << 21, 4, 4, 4), 1), ((40000, 40000, 1, 2), 1)])
def test_plan_rejects_bad_shapes(lib, dims, status):
    h = ctypes.c_void_p()
    st = lib.qtp_plan_create(ctypes.byref(h), *dims, 0, 0)
    assert st == status
    assert h.value is None
    assert len(lib.qtp_last_error()) > 0


def test_plan_rejects_bad_flags_and_precision(lib):
    h = ctypes.c_void_p()
    assert lib.qtp_plan_create(ctypes.byref(h), 4, 4, 4, 4, 0, 4) == 1   # unknown flag bit
    assert lib.qtp_plan_create(ctypes.byref(h), 4, 4, 4, 4, 7, 0) == 1
    assert lib.qtp_plan_create(None, 4, 4, 4, 4, 0, 0) == 1


def test_calls_reject_null_plan(lib):
    sz = ctypes.c_size_t()
    assert lib.qtp_workspace_size(None, ctypes.byref(sz)) == 1
    assert lib.qtp_forward(None, None, None, None, None, 0, None) == 1
    assert lib.qtp_backward(None, None, None, None, None, None, None, 0, None) == 1
    assert lib.qtp_forward_host(None, None, None, None, None, 0, None) == 1
    assert lib.qtp_host_many_buffer_size(None, ctypes.byref(sz)) == 1
    assert lib.qtp_forward_host_many(None, 1, None, None, None, None, 0, None) == 1


def test_tsvd_rejects_bad_shapes_and_pointers(lib):
    sz = ctypes.c_size_t()
    assert lib.qtp_tsvd_workspace_size(0, 4, 4, ctypes.byref(sz)) == 1
    assert lib.qtp_tsvd_workspace_size(4, 4, 5000, ctypes.byref(sz)) == 2
    assert lib.qtp_tsvd_workspace_size(65, 70, 4, ctypes.byref(sz)) == 2      # min(m, n) > 64
    assert lib.qtp_tsvd_workspace_size(8, 2000, 4, ctypes.byref(sz)) == 2     # max(m, n) > 1024
    assert lib.qtp_tsvd_workspace_size(8, 6, 4, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.qtp_tsvd(8, 6, 4, None, None, None, None, None, None, 0, None) == 1
    assert lib.qtp_plan_destroy(None) == 0
