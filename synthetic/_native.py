"""Builds and loads the C half of the synthetic-input generator (gen.c).

The shared object is compiled in-tree with gcc on first use (or by the
repository's build step) and loaded with ctypes.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "libsyngen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into _lib/libsyngen.so if it is missing or stale."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u64, i64, p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        L.syn_stream_key.argtypes = [u64, u64]
        L.syn_stream_key.restype = u64
        L.syn_normal_at.argtypes = [u64, i64, p, p]
        L.syn_normal_at.restype = None
        L.syn_normal_panel.argtypes = [u64, i64, i64, i64, p]
        L.syn_normal_panel.restype = None
        L.syn_sign_panel.argtypes = [u64, i64, i64, i64, p]
        L.syn_sign_panel.restype = None
        L.syn_symmetric_values.argtypes = [u64, i64, p, p, p, p, p, p]
        L.syn_symmetric_values.restype = ctypes.c_int
        _lib = L
    return _lib


def ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data
