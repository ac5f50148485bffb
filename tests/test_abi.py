"""The C-ABI library loads and exports every entry point include/*.h declares,
and host-side argument checks work without a GPU (no compute is run here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1208_3933_gb300 import fsp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fsp_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1208_3933_gb300 import build
    build.build()
    return fsp.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "fsp_bound_pool" in names and "fsp_instance_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(-7, 1):
        assert fsp.fsp_status_string(code)
    assert fsp.fsp_status_string(-5) == "timed out"
    assert fsp.fsp_status_string(99) == "unknown status"
    assert fsp.fsp_version().count(".") == 2


def test_instance_create_rejects_bad_arguments_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    P = ctypes.POINTER(ctypes.c_int32)
    p = np.ones((4, 3), np.int32)
    assert lib.fsp_instance_create(p.ctypes.data_as(P), 0, 3, ctypes.byref(h)) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create(p.ctypes.data_as(P), 4, 1, ctypes.byref(h)) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create(p.ctypes.data_as(P), 1025, 3, ctypes.byref(h)) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create(p.ctypes.data_as(P), 4, 33, ctypes.byref(h)) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create(None, 4, 3, ctypes.byref(h)) == fsp.FSP_EINVAL
    neg = p.copy(); neg[1, 1] = -1
    assert lib.fsp_instance_create(neg.ctypes.data_as(P), 4, 3, ctypes.byref(h)) == fsp.FSP_EINVAL
    big = np.full((4, 3), 2 ** 28, np.int32)  # sum >= 2^30
    assert lib.fsp_instance_create(big.ctypes.data_as(P), 4, 3, ctypes.byref(h)) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create(p.ctypes.data_as(P), 4, 3, None) == fsp.FSP_EINVAL
    assert lib.fsp_instance_create_ex(p.ctypes.data_as(P), 4, 3, 0x2, ctypes.byref(h)) == fsp.FSP_EINVAL


def test_null_handles_are_rejected(lib):
    assert lib.fsp_bound_pool(None, None, None, 0, None, None) == fsp.FSP_EINVAL
    assert lib.fsp_bound_pool_host(None, None, None, 0, None, None) == fsp.FSP_EINVAL
    assert lib.fsp_instance_query(None, None) == fsp.FSP_EINVAL
    assert lib.fsp_branch_and_bound(None, 0, None, None, None) == fsp.FSP_EINVAL
    assert lib.fsp_branch_and_bound_device(None, 0, 0, 0, 0, None, None, None) == fsp.FSP_EINVAL
    lib.fsp_instance_destroy(None)  # no-op
    assert lib.fsp_kernel_launches() >= 0
    assert lib.fsp_check_wait_timeout(None, 1) == fsp.FSP_EINVAL
    assert lib.fsp_server_solve(None, None, 0, 1, 1, 0, None, None, None, None) == fsp.FSP_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(fsp, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(fsp, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        fsp.load()
