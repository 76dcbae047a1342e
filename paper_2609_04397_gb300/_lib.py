"""ctypes binding of libvbcsr.so (the C ABI declared in include/vbcsr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. Loading fails loudly when the library has not been built.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_lib", "libvbcsr.so")

VBCSR_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "PATTERN", -3: "CUDA", -4: "NO_MEMORY",
          -5: "UNSUPPORTED", -6: "DEVICE_CHECK", -7: "ALIAS"}
F64, F32, C128 = 0, 1, 2
PRECISION = {"native": 0, "f32": 1, "tf32": 2, "tf32x3": 3, "bf16x2": 4, "df32": 5}

# every function that include/vbcsr.h declares, with its ctypes signature
_i64, _i32, _d, _p, _int = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int


class Info(ctypes.Structure):
    _fields_ = [("n_brows", _i64), ("n_bcols", _i64), ("n_rows", _i64), ("n_cols", _i64),
                ("nblk", _i64), ("nnz", _i64), ("panel_elems", _i64), ("device_bytes", _i64),
                ("dtype", _i32), ("n_shape_classes", _i32), ("n_row_classes", _i32), ("n_structs", _i32),
                ("backend", _i32), ("reserved", _i32)]


class Epilogue(ctypes.Structure):
    _fields_ = [("gamma", _d), ("Z", _p), ("ldz", _i64), ("R", _p), ("ldr", _i64), ("dot_out", _p)]


SIGNATURES = {
    "vbcsr_error_string": ([_int], ctypes.c_char_p),
    "vbcsr_last_error_detail": ([], ctypes.c_char_p),
    "vbcsr_create": ([ctypes.POINTER(_p), _i64, _i64, _p, _p, _p, _p, _p, _int, _int, _p], _int),
    "vbcsr_create_batched": ([ctypes.POINTER(_p), _i64, _p, _p, _p, _p, _p, _p, _p, _int, _int, _p], _int),
    "vbcsr_destroy": ([_p], _int),
    "vbcsr_set_values": ([_p, _p, _int, _p], _int),
    "vbcsr_get_values": ([_p, _p, _int, _p], _int),
    "vbcsr_spmm": ([_p, _i64, _d, _p, _i64, _d, _p, _i64, _int, _p], _int),
    "vbcsr_spmm_adjoint": ([_p, _i64, _d, _p, _i64, _d, _p, _i64, _int, _p], _int),
    "vbcsr_spmm_ex": ([_p, _int, _i64, _d, _p, _i64, _d, _p, _i64, ctypes.POINTER(Epilogue), _int, _p], _int),
    "vbcsr_sddmm": ([_p, _i64, _d, _p, _i64, _p, _i64, _d, _p, _p], _int),
    "vbcsr_chebyshev": ([_p, _i64, _p, _i64, _i64, _p, _p, _p, _i64, _int, _p], _int),
    "vbcsr_chebyshev_backward": ([_p, _i64, _p, _i64, _i64, _p, _p, _i64, _d, _p, _p, _int, _p], _int),
    "vbcsr_chebyshev_noalloc": ([_p, _i64, _p, _i64, _i64, _p, _int, _p], _int),
    "vbcsr_gershgorin": ([_p, _p, _p], _int),
    "vbcsr_kpm_moments": ([_p, _i64, _p, _i64, _i64, _p, _p, _int, _p], _int),
    "vbcsr_kpm_dos": ([_p, _i64, _int, _p, _i64, _p, _p], _int),
    "vbcsr_kpm_gap": ([_p, _p, _i64, _d, _d, _p, _p], _int),
    "vbcsr_shift_scale": ([_p, _d, _d, _p], _int),
    "vbcsr_spgemm": ([_p, _p, _d, ctypes.POINTER(_p), _p], _int),
    "vbcsr_create_kspace": ([ctypes.POINTER(_p), _i64, _p, _i64, _p, _p, _p, _p, _p, _p], _int),
    "vbcsr_set_kpoint": ([_p, _p, _p], _int),
    "vbcsr_get_info": ([_p, ctypes.POINTER(Info)], _int),
    "vbcsr_get_pattern": ([_p, _p, _p, _p, _p], _int),
    "vbcsr_shape_classes": ([_p, _p, _p, _p, _i32], _int),
    "vbcsr_set_tuning": ([_p, _i32, _i32], _int),
    "vbcsr_set_bucket_tuning": ([_p, _i32, _i32, _i32], _int),
    "vbcsr_set_schedule": ([_p, _i32, _i32], _int),
    "vbcsr_get_tuning": ([_p, _p, _p, _p, _p], _int),
    "vbcsr_autotune": ([_p, _int, _i64, _p, _i64, _p, _i64, _int, _i32, _p], _int),
    "vbcsr_check": ([_p, _p], _int),
}

_lib = None


class VBCSRError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


def lib():
    """Load libvbcsr.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise RuntimeError(f"libvbcsr.so not built ({SO_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(SO_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(status: int, where: str):
    if status < 0:
        raise VBCSRError(status, where, lib().vbcsr_last_error_detail().decode())
    return status
