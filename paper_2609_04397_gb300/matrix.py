"""The VBCSR operator object: a thin PyTorch-facing wrapper of the C ABI.

PyTorch only provides device memory and the current CUDA stream; every
product, permutation and reduction runs in libvbcsr.so.
"""
import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import C128, F32, F64, PRECISION, check, lib

_TORCH_DTYPE = {F64: torch.float64, F32: torch.float32, C128: torch.complex128}
_CODE = {torch.float64: F64, torch.float32: F32, torch.complex128: C128}
_NP = {torch.float64: np.float64, torch.float32: np.float32, torch.complex128: np.complex128}


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _np(a, dt):
    return np.ascontiguousarray(np.asarray(a), dtype=dt)


def _cuda_device(device) -> torch.device:
    """The CUDA device a new operator lives on, with its index made explicit
    ("cuda" means the current device), so that tensors created on it compare
    equal to it."""
    dev = torch.device(device or "cuda")
    if dev.type != "cuda":
        raise ValueError(f"operators live on a CUDA device, not {dev}")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    return dev


def _prec(precision) -> int:
    if isinstance(precision, int):
        return precision
    return PRECISION[precision.lower()]


class VBCSR:
    """A variable-block sparse operator resident on one GPU (Sec. II.A)."""

    def __init__(self, handle: ctypes.c_void_p, dtype: int, device: torch.device, pattern):
        self._h = handle
        self._dtype = dtype
        self.device = device
        self.pattern = pattern           # (row_bsize, col_bsize, block_row_ptr, block_col_idx) as numpy
        info = _lib.Info()
        check(lib().vbcsr_get_info(self._h, ctypes.byref(info)), "vbcsr_get_info")
        self.info = info

    # ---- construction ---------------------------------------------------

    @classmethod
    def from_arrays(cls, row_bsize, col_bsize, block_row_ptr, block_col_idx, values,
                    dtype: torch.dtype = torch.float64, device=None) -> "VBCSR":
        """Build from host pattern arrays and packed values (numpy array or
        torch tensor, host or device), blocks row-major in pattern order."""
        device = _cuda_device(device)
        dt = _CODE[dtype]
        rb, cb = _np(row_bsize, np.int32), _np(col_bsize, np.int32)
        rp, ci = _np(block_row_ptr, np.int64), _np(block_col_idx, np.int32)
        on_dev, vptr, keep = cls._values_arg(values, dtype, device)
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            check(lib().vbcsr_create(ctypes.byref(h), len(rb), len(cb), rb.ctypes.data, cb.ctypes.data,
                                     rp.ctypes.data, ci.ctypes.data, vptr, dt, on_dev, _stream(device)),
                  "vbcsr_create")
        del keep
        return cls(h, dt, device, (rb, cb, rp, ci))

    @classmethod
    def from_pattern(cls, pattern, values, dtype=torch.float64, device=None) -> "VBCSR":
        return cls.from_arrays(pattern.row_bsize, pattern.col_bsize, pattern.block_row_ptr,
                               pattern.block_col_idx, values, dtype, device)

    @classmethod
    def from_batched(cls, struct_brow_offsets, struct_bcol_offsets, row_bsize, col_bsize,
                     block_row_ptr, local_block_col_idx, values, dtype=torch.float64, device=None) -> "VBCSR":
        """One operator over independent structures; column indices local to
        each structure (see vbcsr_create_batched)."""
        device = _cuda_device(device)
        dt = _CODE[dtype]
        so, co = _np(struct_brow_offsets, np.int64), _np(struct_bcol_offsets, np.int64)
        rb, cb = _np(row_bsize, np.int32), _np(col_bsize, np.int32)
        rp, ci = _np(block_row_ptr, np.int64), _np(local_block_col_idx, np.int32)
        on_dev, vptr, keep = cls._values_arg(values, dtype, device)
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            check(lib().vbcsr_create_batched(ctypes.byref(h), len(so) - 1, so.ctypes.data, co.ctypes.data,
                                             rb.ctypes.data, cb.ctypes.data, rp.ctypes.data, ci.ctypes.data,
                                             vptr, dt, on_dev, _stream(device)), "vbcsr_create_batched")
        del keep
        gcol = ci.astype(np.int64).copy()
        rows = np.repeat(np.arange(len(rb)), np.diff(rp))
        s_of_row = np.searchsorted(so, rows, side="right") - 1
        gcol += co[s_of_row]
        return cls(h, dt, device, (rb, cb, rp, gcol.astype(np.int32)))

    @classmethod
    def from_images(cls, bsize, edge_i, edge_j, edge_R, edge_values, tau=None, device=None) -> "VBCSR":
        """A periodic operator sampled in reciprocal space (Eq. 4, see
        vbcsr_create_kspace): edges (i, j, R) of the real-space images with
        their real b_i x b_j blocks packed row-major in edge order (numpy);
        tau: fractional atom positions for the R+tau convention, or None.
        The result is complex128 and zero until set_kpoint."""
        device = _cuda_device(device)
        bs = _np(bsize, np.int32)
        ei, ej = _np(edge_i, np.int32), _np(edge_j, np.int32)
        eR = _np(edge_R, np.int32).reshape(-1, 3)
        ev = _np(edge_values, np.float64)
        tp = _np(tau, np.float64).reshape(-1, 3) if tau is not None else None
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            check(lib().vbcsr_create_kspace(ctypes.byref(h), len(bs), bs.ctypes.data, len(ei), ei.ctypes.data,
                                            ej.ctypes.data, eR.ctypes.data, ev.ctypes.data,
                                            tp.ctypes.data if tp is not None else None, _stream(device)),
                  "vbcsr_create_kspace")
        H = cls(h, C128, device, None)
        H.pattern = H.read_pattern()
        return H

    def set_kpoint(self, kfrac):
        """Fill a from_images operator with O(k), k in fractional reciprocal coordinates."""
        k = np.ascontiguousarray(np.asarray(kfrac, dtype=np.float64).reshape(3))
        check(lib().vbcsr_set_kpoint(self._h, k.ctypes.data, _stream(self.device)), "vbcsr_set_kpoint")

    @staticmethod
    def _values_arg(values, dtype, device):
        if isinstance(values, torch.Tensor):
            if values.dtype != dtype:
                raise TypeError(f"values dtype {values.dtype} != {dtype}")
            v = values.contiguous()
            if v.is_cuda:
                return 1, v.data_ptr(), v
            return 0, v.data_ptr(), v
        v = np.ascontiguousarray(values, dtype=_NP[dtype])
        return 0, v.ctypes.data, v

    def close(self):
        if getattr(self, "_h", None):
            lib().vbcsr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- properties -----------------------------------------------------

    @property
    def dtype(self) -> torch.dtype:
        return _TORCH_DTYPE[self._dtype]

    @property
    def shape(self):
        return (int(self.info.n_rows), int(self.info.n_cols))

    @property
    def backend(self) -> str:
        """'csr', 'bsr' or 'vbcsr' (chosen from the block sizes)."""
        return ("csr", "bsr", "vbcsr")[self.info.backend]

    @property
    def nnz(self) -> int:
        return int(self.info.nnz)

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def shape_classes(self):
        """[(b_i, b_j, count)] from the shape-class registry."""
        n = check(lib().vbcsr_shape_classes(self._h, None, None, None, 0), "vbcsr_shape_classes")
        bi = np.zeros(n, np.int32)
        bj = np.zeros(n, np.int32)
        cnt = np.zeros(n, np.int64)
        check(lib().vbcsr_shape_classes(self._h, bi.ctypes.data, bj.ctypes.data, cnt.ctypes.data, n),
              "vbcsr_shape_classes")
        return list(zip(bi.tolist(), bj.tolist(), cnt.tolist()))

    def set_tuning(self, kc: int = 0, warps: int = 0, B: int = 0):
        """Column tile and CTA width of the bucket of row count B (0: all)."""
        check(lib().vbcsr_set_bucket_tuning(self._h, B, kc, warps), "vbcsr_set_bucket_tuning")

    def set_schedule(self, schedule: str = "persistent", persist_warps: int = 0, mma_staged: bool = False,
                     scalar_kernel: bool = True, value_ring: bool = True, pipelined_f32: bool = True):
        """'persistent' (one launch over every item, the default) or 'bucketed'
        (one launch per row count);
        mma_staged selects the shared-memory-staged tensor-core forward kernel;
        scalar_kernel=False makes a CSR-backend operator use the block-row kernels;
        value_ring=False makes the FP32-value CUDA-core forward kernel read its
        values directly instead of through its shared-memory ring (k >= 8);
        pipelined_f32=False makes the persistent launch on FP32 values at k >= 8
        use that kernel instead of the pipelined one."""
        code = ({"bucketed": 0, "persistent": 1}[schedule] | (2 if mma_staged else 0)
                | (0 if scalar_kernel else 4) | (0 if value_ring else 8) | (0 if pipelined_f32 else 16))
        check(lib().vbcsr_set_schedule(self._h, code, persist_warps), "vbcsr_set_schedule")

    def get_tuning(self) -> dict:
        kc = np.zeros(17, np.int32)
        w = np.zeros(17, np.int32)
        sch = ctypes.c_int32()
        pw = ctypes.c_int32()
        check(lib().vbcsr_get_tuning(self._h, kc.ctypes.data, w.ctypes.data, ctypes.byref(sch),
                                     ctypes.byref(pw)), "vbcsr_get_tuning")
        return {"kc_by_b": kc.tolist(), "warps_by_b": w.tolist(),
                "schedule": ["bucketed", "persistent"][sch.value & 1], "mma_staged": bool(sch.value & 2),
                "scalar_kernel": not (sch.value & 4), "value_ring": not (sch.value & 8),
                "pipelined_f32": not (sch.value & 16), "persist_warps": pw.value}

    def apply_tuning(self, t: dict):
        for B in range(1, 17):
            self.set_tuning(t["kc_by_b"][B], t["warps_by_b"][B], B)
        self.set_schedule(t["schedule"], t["persist_warps"], t.get("mma_staged", False),
                          t.get("scalar_kernel", True), t.get("value_ring", True), t.get("pipelined_f32", True))

    def autotune(self, k: int, precision="native", transpose: bool = False, allow_persistent: bool = True,
                 cache: Optional[str] = None) -> dict:
        """Choose per-row-count tiles and the schedule by timing the product at
        width k on scratch panels; with `cache`, reuse/record the choice in a
        JSON file keyed by the pattern, k, precision and direction."""
        key = None
        if cache:
            import hashlib
            import json
            import os
            h = hashlib.sha1()
            for a in self.pattern:
                h.update(np.ascontiguousarray(a).tobytes())
            key = f"{h.hexdigest()}:{k}:{precision}:{int(transpose)}:{int(allow_persistent)}"
            if os.path.exists(cache):
                with open(cache) as f:
                    db = json.load(f)
                if key in db:
                    self.apply_tuning(db[key])
                    return db[key]
        n_in, n_out = (self.shape[0], self.shape[1]) if transpose else (self.shape[1], self.shape[0])
        X = torch.randn(n_in, k, dtype=self.dtype, device=self.device)
        Y = torch.empty(n_out, k, dtype=self.dtype, device=self.device)
        check(lib().vbcsr_autotune(self._h, int(transpose), k, ctypes.c_void_p(X.data_ptr()), k,
                                   ctypes.c_void_p(Y.data_ptr()), k, _prec(precision),
                                   0 if allow_persistent else 1, _stream(self.device)), "vbcsr_autotune")
        t = self.get_tuning()
        if cache:
            import json
            import os
            db = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    db = json.load(f)
            db[key] = t
            with open(cache, "w") as f:
                json.dump(db, f)
        return t

    def check(self):
        check(lib().vbcsr_check(self._h, _stream(self.device)), "vbcsr_check")

    # ---- values ----------------------------------------------------------

    def set_values(self, values):
        on_dev, vptr, keep = self._values_arg(values, self.dtype, self.device)
        check(lib().vbcsr_set_values(self._h, vptr, on_dev, _stream(self.device)), "vbcsr_set_values")
        if on_dev:
            # the tensor must stay alive until the scatter has run on the stream
            keep.record_stream(torch.cuda.current_stream(self.device))

    def get_values(self) -> torch.Tensor:
        out = torch.empty(self.nnz, dtype=self.dtype, device=self.device)
        check(lib().vbcsr_get_values(self._h, ctypes.c_void_p(out.data_ptr()), 1, _stream(self.device)),
              "vbcsr_get_values")
        return out

    # ---- products --------------------------------------------------------

    def _panel(self, T: torch.Tensor, rows: int, name: str):
        if not isinstance(T, torch.Tensor) or T.device != self.device or T.dtype != self.dtype:
            raise TypeError(f"{name} must be a {self.dtype} tensor on {self.device}")
        if T.dim() == 1:
            T = T.view(-1, 1)
        if T.dim() != 2 or T.shape[0] != rows or (T.shape[1] > 1 and T.stride(1) != 1):
            raise ValueError(f"{name} must be a row-major [{rows}, k] panel, got {tuple(T.shape)} "
                             f"strides {T.stride()}")
        ld = T.stride(0) if T.shape[1] > 1 or T.shape[0] > 1 else 1
        return T, max(ld, T.shape[1])

    def _prod(self, transpose: bool, X, alpha, beta, Y, precision, epilogue=None):
        n_out, n_in = (self.shape[1], self.shape[0]) if transpose else self.shape
        squeeze = X.dim() == 1
        X, ldx = self._panel(X, n_in, "X")
        k = X.shape[1]
        if Y is None:
            Y = torch.empty((n_out, k), dtype=self.dtype, device=self.device)
            beta = 0.0
        Y2, ldy = self._panel(Y, n_out, "Y")
        if Y2.shape[1] != k:
            raise ValueError("X and Y have different column counts")
        if epilogue is None:
            fn = lib().vbcsr_spmm_adjoint if transpose else lib().vbcsr_spmm
            check(fn(self._h, k, float(alpha), ctypes.c_void_p(X.data_ptr()), ldx, float(beta),
                     ctypes.c_void_p(Y2.data_ptr()), ldy, _prec(precision), _stream(self.device)),
                  "vbcsr_spmm_adjoint" if transpose else "vbcsr_spmm")
        else:
            check(lib().vbcsr_spmm_ex(self._h, int(transpose), k, float(alpha), ctypes.c_void_p(X.data_ptr()),
                                      ldx, float(beta), ctypes.c_void_p(Y2.data_ptr()), ldy,
                                      ctypes.byref(epilogue), _prec(precision), _stream(self.device)),
                  "vbcsr_spmm_ex")
        return Y.view(-1) if squeeze and Y.dim() == 1 else Y

    def spmm(self, X, alpha=1.0, beta=0.0, Y=None, precision="native"):
        """Y = alpha H X + beta Y (a new Y when Y is None)."""
        return self._prod(False, X, alpha, beta, Y, precision)

    def spmm_adjoint(self, X, alpha=1.0, beta=0.0, Y=None, precision="native"):
        """Y = alpha H^dagger X + beta Y (Eq. 1): the transpose of a real operator,
        the conjugate transpose of a complex one."""
        return self._prod(True, X, alpha, beta, Y, precision)

    def spmm_ex(self, X, alpha, beta, Y, transpose=False, gamma=0.0, Z=None, R=None,
                dot_out: Optional[torch.Tensor] = None, precision="native"):
        """Y = alpha op(H) X + beta Y + gamma Z; dot_out[0] = sum(R * Y)."""
        epi = _lib.Epilogue()
        epi.gamma = float(gamma)
        if gamma != 0.0:
            Zp, epi.ldz = self._panel(Z, Y.shape[0], "Z")
            epi.Z = Zp.data_ptr()
        if dot_out is not None:
            Rp, epi.ldr = self._panel(R, Y.shape[0], "R")
            epi.R = Rp.data_ptr()
            assert dot_out.dtype == torch.float64 and dot_out.is_cuda
            epi.dot_out = dot_out.data_ptr()
        return self._prod(transpose, X, alpha, beta, Y, precision, epi)

    def sddmm(self, A, B, alpha=1.0, beta=0.0, D=None):
        """D_ij = alpha A[rows_i] B[cols_j]^T + beta D_ij on the stored blocks,
        packed order (the gradient of <A, H B> with respect to the values)."""
        A, lda = self._panel(A, self.shape[0], "A")
        B, ldb = self._panel(B, self.shape[1], "B")
        if A.shape[1] != B.shape[1]:
            raise ValueError("A and B have different column counts")
        if D is None:
            D = torch.empty(self.nnz, dtype=self.dtype, device=self.device)
            beta = 0.0
        check(lib().vbcsr_sddmm(self._h, A.shape[1], float(alpha), ctypes.c_void_p(A.data_ptr()), lda,
                                ctypes.c_void_p(B.data_ptr()), ldb, float(beta), ctypes.c_void_p(D.data_ptr()),
                                _stream(self.device)), "vbcsr_sddmm")
        return D

    def chebyshev(self, R, n_moments: int, ckpt_every: int = 0, precision="native"):
        """Moments mu_n = Re <R, T_n(H) R> / (N k) of an operator already scaled
        to [-1, 1] (R in the operator's dtype: complex for a complex Hermitian
        operator); returns (moments, checkpoints or None)."""
        R, ldr = self._panel(R, self.shape[0], "R")
        k = R.shape[1]
        N = self.shape[0]
        mom = torch.empty(n_moments, dtype=torch.float64, device=self.device)
        work = torch.empty(2 * N * k, dtype=self.dtype, device=self.device)
        ck = None
        if ckpt_every:
            npairs = max(0, -(-(n_moments - 1) // ckpt_every))
            ck = torch.empty((npairs, 2, N, k), dtype=self.dtype, device=self.device)
        check(lib().vbcsr_chebyshev(self._h, k, ctypes.c_void_p(R.data_ptr()), ldr, n_moments,
                                    ctypes.c_void_p(mom.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                    ctypes.c_void_p(ck.data_ptr() if ck is not None else None),
                                    ckpt_every, _prec(precision), _stream(self.device)), "vbcsr_chebyshev")
        return mom, ck

    def kpm_moments(self, R, n_moments: int, precision="native"):
        """KPM moments of a symmetric (or complex Hermitian) operator scaled to
        [-1, 1], by the doubling identities (about half the products of
        chebyshev())."""
        R, ldr = self._panel(R, self.shape[0], "R")
        k = R.shape[1]
        mom = torch.empty(n_moments, dtype=torch.float64, device=self.device)
        work = torch.empty(2 * self.shape[0] * k, dtype=self.dtype, device=self.device)
        check(lib().vbcsr_kpm_moments(self._h, k, ctypes.c_void_p(R.data_ptr()), ldr, n_moments,
                                      ctypes.c_void_p(mom.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                      _prec(precision), _stream(self.device)), "vbcsr_kpm_moments")
        return mom

    def spgemm(self, other: "VBCSR", eps: float = 0.0) -> "VBCSR":
        """C = self @ other with the block-norm threshold eps (Eqs. 2-3)."""
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().vbcsr_spgemm(self._h, other._h, float(eps), ctypes.byref(h), _stream(self.device)),
                  "vbcsr_spgemm")
        C = VBCSR(h, self._dtype, self.device, None)
        C.pattern = C.read_pattern()
        return C

    def read_pattern(self):
        """(row_bsize, col_bsize, block_row_ptr, block_col_idx) held by the handle."""
        i = self.info
        rb = np.zeros(i.n_brows, np.int32)
        cb = np.zeros(i.n_bcols, np.int32)
        rp = np.zeros(i.n_brows + 1, np.int64)
        ci = np.zeros(i.nblk, np.int32)
        check(lib().vbcsr_get_pattern(self._h, rb.ctypes.data, cb.ctypes.data, rp.ctypes.data, ci.ctypes.data),
              "vbcsr_get_pattern")
        return rb, cb, rp, ci

    def gershgorin(self):
        """(E_min, E_max): Gershgorin bounds of the spectrum, computed on the GPU."""
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        check(lib().vbcsr_gershgorin(self._h, ctypes.c_void_p(out.data_ptr()), _stream(self.device)),
              "vbcsr_gershgorin")
        lo, hi = out.tolist()
        return lo, hi

    def shift_scale(self, c: float, d: float):
        """Values <- (H - c I) / d in place."""
        check(lib().vbcsr_shift_scale(self._h, float(c), float(d), _stream(self.device)), "vbcsr_shift_scale")

    def __matmul__(self, X):
        return self.spmm(X)


def kpm_dos(moments: torch.Tensor, x: torch.Tensor, kernel: str = "jackson") -> torch.Tensor:
    """Density of states at scaled energies x (device tensors, FP64) from KPM
    moments, with Jackson damping (kernel='jackson') or none ('none')."""
    moments = moments.contiguous()
    x = x.contiguous()
    out = torch.empty_like(x)
    code = {"none": 0, "jackson": 1}[kernel]
    check(lib().vbcsr_kpm_dos(ctypes.c_void_p(moments.data_ptr()), moments.numel(), code,
                              ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(out.data_ptr()),
                              _stream(x.device)), "vbcsr_kpm_dos")
    return out


def kpm_gap(energies: torch.Tensor, dos: torch.Tensor, reference: float, threshold: float):
    """Band gap read off a density of states on an energy grid (device FP64
    tensors, energies increasing; see vbcsr_kpm_gap): the widest run of grid
    points around the one nearest `reference` whose DOS stays below
    `threshold`, as (E_low, E_high), or None when the reference lies inside a
    band. The search runs in the library; only the two energies come back."""
    energies = energies.contiguous()
    dos = dos.contiguous()
    if energies.shape != dos.shape or energies.dim() != 1:
        raise ValueError("energies and dos must be 1-D tensors of one length")
    out = torch.empty(2, dtype=torch.float64, device=energies.device)
    check(lib().vbcsr_kpm_gap(ctypes.c_void_p(energies.data_ptr()), ctypes.c_void_p(dos.data_ptr()),
                              energies.numel(), float(reference), float(threshold), ctypes.c_void_p(out.data_ptr()),
                              _stream(energies.device)), "vbcsr_kpm_gap")
    lo, hi = out.tolist()
    if lo != lo:
        return None
    return lo, hi
