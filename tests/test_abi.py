"""The C ABI library loads, exports what include/vbcsr.h declares, and rejects
invalid input on the host before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vbcsr_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2609_04397_gb300 import build
    build.build()
    from paper_2609_04397_gb300 import _lib
    return _lib.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert {"vbcsr_create", "vbcsr_spmm", "vbcsr_spmm_adjoint", "vbcsr_destroy"} <= names
    for n in names:
        assert hasattr(L, n), n
    from paper_2609_04397_gb300 import _lib
    assert names == set(_lib.SIGNATURES), "binding and header disagree"


def test_error_strings(L):
    for code in range(0, -8, -1):
        s = L.vbcsr_error_string(code)
        assert s and s != b"unknown status"
    assert L.vbcsr_error_string(-99) == b"unknown status"


def _create(L, rb, cb, rp, ci, vals, dtype=0):
    rb = np.ascontiguousarray(rb, np.int32)
    cb = np.ascontiguousarray(cb, np.int32)
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    v = np.ascontiguousarray(vals, np.float64)
    h = ctypes.c_void_p()
    rc = L.vbcsr_create(ctypes.byref(h), len(rb), len(cb), rb.ctypes.data, cb.ctypes.data, rp.ctypes.data,
                        ci.ctypes.data if len(ci) else None, v.ctypes.data, dtype, 0, None)
    return rc, h, L.vbcsr_last_error_detail().decode()


@pytest.mark.parametrize("case,expect,needle", [
    (dict(rp=[1, 2, 3]), -2, "block_row_ptr[0]"),
    (dict(rp=[0, 2, 1]), -2, "decreases"),
    (dict(ci=[0, 2, 1]), -2, "outside"),
    (dict(ci=[0, 0, 1]), -2, "duplicate"),
    (dict(rp=[0, 3, 4], ci=[1, 0, 1, 1]), -2, "duplicate"),   # unsorted row with a duplicate
    (dict(rp=[0, 3, 4], ci=[1, 0, 2, 1]), -2, "outside"),
    (dict(ci=[0, -1, 1]), -2, "outside"),
    (dict(rb=[0, 2]), -2, "row_bsize"),
    (dict(cb=[1, 5000]), -2, "col_bsize"),
    (dict(dtype=7), -1, "dtype"),
])
def test_host_validation_rejects_bad_patterns(L, case, expect, needle):
    args = dict(rb=[1, 2], cb=[1, 2], rp=[0, 2, 3], ci=[0, 1, 1], vals=np.ones(1 + 2 + 4))
    args.update(case)
    rc, h, detail = _create(L, args["rb"], args["cb"], args["rp"], args["ci"], args["vals"],
                            args.get("dtype", 0))
    assert rc == expect, detail
    assert needle in detail
    assert not h.value


def test_null_arguments_rejected(L):
    rc = L.vbcsr_create(None, 0, 0, None, None, None, None, None, 0, 0, None)
    assert rc == -1
    assert L.vbcsr_spmm(None, 1, 1.0, None, 1, 0.0, None, 1, 0, None) == -1
    assert L.vbcsr_destroy(None) == 0


def test_valid_pattern_without_gpu_reports_cuda_error(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    rc, h, detail = _create(L, [1, 2], [1, 2], [0, 2, 3], [0, 1, 1], np.ones(7))
    assert rc in (-3, -4), detail      # validation passed; the device is what is missing
    assert not h.value


def test_product_failure_modes_are_compiled_in(L):
    """The binding raises a VBCSRError with the library's detail message."""
    from paper_2609_04397_gb300._lib import VBCSRError, check
    with pytest.raises(VBCSRError) as ei:
        check(L.vbcsr_set_tuning(None, 8, 4), "vbcsr_set_tuning")
    assert "INVALID_ARG" in str(ei.value)


def test_kspace_host_validation(L):
    """vbcsr_create_kspace rejects bad edges on the host; vbcsr_set_kpoint
    rejects NULL handles and k-points."""
    from paper_2609_04397_gb300._lib import SIGNATURES  # noqa: F401 (signatures set on load)
    h = ctypes.c_void_p()
    bs = np.array([2, 3], np.int32)
    ei, ej = np.array([0, 1], np.int32), np.array([1, 2], np.int32)     # atom 2 does not exist
    eR = np.zeros((2, 3), np.int32)
    ev = np.ones(12)
    rc = L.vbcsr_create_kspace(ctypes.byref(h), 2, bs.ctypes.data, 2, ei.ctypes.data, ej.ctypes.data,
                               eR.ctypes.data, ev.ctypes.data, None, None)
    assert rc == -2 and not h.value
    assert b"outside" in L.vbcsr_last_error_detail()
    bad = np.array([2, 0], np.int32)                                    # block size 0
    ej_ok = np.array([1, 0], np.int32)
    rc = L.vbcsr_create_kspace(ctypes.byref(h), 2, bad.ctypes.data, 2, ei.ctypes.data, ej_ok.ctypes.data,
                               eR.ctypes.data, ev.ctypes.data, None, None)
    assert rc == -2
    rc = L.vbcsr_create_kspace(ctypes.byref(h), 2, bs.ctypes.data, 2, None, ej_ok.ctypes.data,
                               eR.ctypes.data, ev.ctypes.data, None, None)
    assert rc == -1
    assert L.vbcsr_set_kpoint(None, None, None) == -1
