"""Python binding of libspc5 (include/spc5.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module turns torch
CUDA tensors into device pointers and the current torch stream into a
cudaStream_t. There is no fallback: if libspc5.so is missing or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

SPC5_F64, SPC5_F32, SPC5_BF16 = 0, 1, 2
STATUS = {0: "SPC5_OK", 1: "SPC5_EINVAL", 2: "SPC5_EUNSORTED", 3: "SPC5_EDUP", 4: "SPC5_ERANGE",
          5: "SPC5_EUNSUPPORTED", 6: "SPC5_ENOMEM", 7: "SPC5_ECUDA", 8: "SPC5_ETIMEOUT"}
OK, EINVAL, EUNSORTED, EDUP, ERANGE, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT = range(9)

_VALUE_DTYPE = {torch.float64: SPC5_F64, torch.float32: SPC5_F32, torch.bfloat16: SPC5_BF16}
_VECTOR_DTYPE = {SPC5_F64: torch.float64, SPC5_F32: torch.float32, SPC5_BF16: torch.float32}
SHAPES = [(r, c) for r in (1, 2, 4, 8) for c in (4, 8, 16)]


class Spc5Error(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("long_blocks", ctypes.c_int32), ("seg_blocks", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("order_window", ctypes.c_int32), ("long_values", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class CgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("inner_max_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("reliable", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class CgInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("inner_total", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


NFEATURES, NFORMATS = 16, 12
SELECT_EXHAUSTIVE, SELECT_POLY, SELECT_MLP = 0, 1, 2


class Selector(ctypes.Structure):
    _fields_ = [("poly_degree", ctypes.c_int32), ("poly_coef", ctypes.c_void_p), ("mlp_params_d", ctypes.c_void_p),
                ("feat_mean", ctypes.c_float * NFEATURES), ("feat_scale", ctypes.c_float * NFEATURES)]


class TuneResult(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("c", ctypes.c_int32), ("variant", ctypes.c_int32), ("spmv_ms", ctypes.c_float),
                ("spmm_r", ctypes.c_int32), ("spmm_c", ctypes.c_int32), ("ktile", ctypes.c_int32),
                ("spmm_ms", ctypes.c_float), ("from_cache", ctypes.c_int32), ("spmm_variant", ctypes.c_int32),
                ("signature", ctypes.c_uint64)]


TUNE_NO_CACHE = 1


class Arrays(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nblocks", ctypes.c_int64),
                ("nintervals", ctypes.c_int64), ("r", ctypes.c_int32), ("c", ctypes.c_int32),
                ("mask_bytes", ctypes.c_int32), ("dtype", ctypes.c_int), ("block_rowptr_d", ctypes.c_void_p),
                ("block_colidx_d", ctypes.c_void_p), ("block_masks_d", ctypes.c_void_p),
                ("values_d", ctypes.c_void_p), ("valptr_d", ctypes.c_void_p), ("nsegments", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libspc5.so (fails loudly when it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is not built; run __graft_entry__.build() (no CPU fallback exists)")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    st = ctypes.c_int
    lib.spc5_convert.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, i32, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.spc5_spmv.argtypes = [vp, vp, vp, vp]
    lib.spc5_spmv_acc.argtypes = [vp, vp, vp, vp]
    lib.spc5_export.argtypes = [vp, ctypes.POINTER(Arrays)]
    lib.spc5_set_variant.argtypes = [vp, i32, vp]
    lib.spc5_autotune.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), vp]
    lib.spc5_destroy.argtypes = [vp]
    lib.spc5_last_error.argtypes = []
    lib.spc5_last_error.restype = ctypes.c_char_p
    lib.spc5_count_blocks.argtypes = [i64, i64, i64, vp, vp, vp, vp]
    lib.spc5_csr_spmv.argtypes = [i64, i64, i64, vp, vp, vp, i32, vp, vp, i32, vp]
    lib.spc5_copy.argtypes = [vp, vp, i64, vp]
    lib.spc5_assemble.argtypes = [i64, i64, i64, i64, vp, vp, vp, vp, i32, i32, i32, ctypes.POINTER(Opts), vp,
                                  ctypes.POINTER(vp)]
    lib.spc5_fma_rate.argtypes = [i32, i64, vp, vp, vp]
    lib.spc5_fma_rate_lanes.argtypes = [i32, i64, i32, vp, vp, vp]
    lib.spc5_spmv_noalloc.argtypes = [vp, vp, vp, vp]
    lib.spc5_launch_count.argtypes = [vp, ctypes.POINTER(i32)]
    lib.spc5_pool_trim.argtypes = []
    lib.spc5_poly2_fit.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.spc5_poly2_select.argtypes = [vp, i32, vp, ctypes.c_double, ctypes.POINTER(i32), ctypes.POINTER(i32), vp]
    lib.spc5_sm_stream_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i32)]
    lib.spc5_sm_stream_destroy.argtypes = [vp]
    lib.spc5_csr_plan_create.argtypes = [i64, i64, vp, i32, i32, i64, i64, vp, ctypes.POINTER(vp)]
    lib.spc5_csr_spmv_plan.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.spc5_csr_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.spc5_csr_plan_destroy.argtypes = [vp]
    lib.spc5_convert_rows.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, i32, i64, i64, ctypes.POINTER(Opts), vp,
                                      ctypes.POINTER(vp)]
    lib.spc5_tune.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, i32, i32, ctypes.POINTER(TuneResult), vp]
    lib.spc5_tune_cache_clear.argtypes = []
    lib.spc5_device_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.spc5_cg.argtypes = [vp, vp, vp, vp, ctypes.POINTER(CgOpts), ctypes.POINTER(CgInfo), vp]
    lib.spc5_spmm.argtypes = [vp, i32, vp, i64, vp, i64, i32, vp]
    lib.spc5_features.argtypes = [i64, i64, i64, vp, vp, vp, vp]
    lib.spc5_batch_create.argtypes = [vp, vp, vp, i32, ctypes.POINTER(vp)]
    lib.spc5_batch_spmv.argtypes = [vp, vp]
    lib.spc5_batch_spmv_direct.argtypes = [vp, vp]
    lib.spc5_batch_destroy.argtypes = [vp]
    lib.spc5_time_formats.argtypes = [i64, i64, i64, vp, vp, vp, i32, vp, vp, i32, vp, vp]
    lib.spc5_mlp_nparams.argtypes = []
    lib.spc5_mlp_nparams.restype = i32
    lib.spc5_mlp_nparams_n.argtypes = [i32]
    lib.spc5_mlp_nparams_n.restype = i32
    lib.spc5_features_ext.argtypes = [i64, i64, i64, vp, vp, ctypes.c_double, vp, vp]
    lib.spc5_mlp_train_n.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]
    lib.spc5_mlp_grad_n.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp]
    lib.spc5_mlp_infer_n.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.spc5_mlp_train.argtypes = [vp, vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]
    lib.spc5_mlp_grad.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    lib.spc5_mlp_infer.argtypes = [vp, vp, i32, vp, vp]
    lib.spc5_poly_fit.argtypes = [vp, vp, i32, i32, vp]
    lib.spc5_partition.argtypes = [vp, i64, i32, vp]
    lib.spc5_select.argtypes = [i64, i64, i64, vp, vp, vp, i32, i32, ctypes.POINTER(Selector), vp, vp, vp, vp]
    for f in (lib.spc5_convert, lib.spc5_assemble, lib.spc5_autotune, lib.spc5_spmv, lib.spc5_spmv_acc, lib.spc5_export, lib.spc5_destroy, lib.spc5_set_variant,
              lib.spc5_count_blocks, lib.spc5_csr_spmv, lib.spc5_copy, lib.spc5_fma_rate, lib.spc5_fma_rate_lanes,
              lib.spc5_spmv_noalloc, lib.spc5_launch_count, lib.spc5_device_peaks, lib.spc5_tune,
              lib.spc5_tune_cache_clear, lib.spc5_convert_rows, lib.spc5_pool_trim, lib.spc5_csr_plan_create,
              lib.spc5_csr_spmv_plan, lib.spc5_csr_plan_info, lib.spc5_csr_plan_destroy, lib.spc5_sm_stream_create,
              lib.spc5_sm_stream_destroy, lib.spc5_poly2_fit, lib.spc5_poly2_select, lib.spc5_features_ext,
              lib.spc5_mlp_train_n, lib.spc5_mlp_grad_n, lib.spc5_mlp_infer_n, lib.spc5_cg, lib.spc5_spmm, lib.spc5_features,
              lib.spc5_time_formats, lib.spc5_mlp_train, lib.spc5_mlp_grad, lib.spc5_mlp_infer, lib.spc5_poly_fit,
              lib.spc5_select, lib.spc5_batch_create, lib.spc5_batch_spmv, lib.spc5_batch_spmv_direct,
              lib.spc5_batch_destroy, lib.spc5_partition):
        f.restype = st
    _lib = lib
    return lib


def last_error() -> str:
    return load().spc5_last_error().decode()


def _check(status: int, where: str):
    if status != OK:
        raise Spc5Error(status, where, last_error())


def _stream_ptr(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr() if t.numel() > 0 else None


def _pad16(nbytes: int) -> int:
    return (nbytes + 15) // 16 * 16 + 16


class Matrix:
    """A matrix converted to beta(r,c); owns the library handle."""

    def __init__(self, handle: int, n: int, m: int, nnz: int, r: int, c: int, vt: int):
        self._h = handle
        self.n, self.m, self.nnz, self.r, self.c, self.vt = n, m, nnz, r, c, vt
        self.variant = 0

    @property
    def vector_dtype(self) -> torch.dtype:
        return _VECTOR_DTYPE[self.vt]

    def spmv(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = A x (overwrites y; allocates it when None)."""
        if y is None:
            y = torch.empty(self.n, dtype=self.vector_dtype, device=x.device)
        self._check_vectors(x, y)
        _check(load().spc5_spmv(self._h, _ptr(x), _ptr(y), _stream_ptr(stream)), "spc5_spmv")
        return y

    def spmv_noalloc(self, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        """y = A x without any allocation by the library (fixed scratch array; see spc5.h)."""
        self._check_vectors(x, y)
        _check(load().spc5_spmv_noalloc(self._h, _ptr(x), _ptr(y), _stream_ptr(stream)), "spc5_spmv_noalloc")
        return y

    def spmv_acc(self, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        """y += A x (the paper's accumulate form)."""
        self._check_vectors(x, y)
        _check(load().spc5_spmv_acc(self._h, _ptr(x), _ptr(y), _stream_ptr(stream)), "spc5_spmv_acc")
        return y

    def _check_vectors(self, x, y):
        if self._h is None:
            raise ValueError("matrix was destroyed")
        if x.dtype != self.vector_dtype or y.dtype != self.vector_dtype:
            raise TypeError(f"x and y must be {self.vector_dtype}")
        if x.numel() != self.m or y.numel() != self.n:
            raise ValueError("x must have m entries and y n entries")

    def spmm(self, X: torch.Tensor, Y: torch.Tensor | None = None, ktile: int = 0, stream=None) -> torch.Tensor:
        """Y = A X for row-major X (m x k) with unit column stride; returns Y (n x k)."""
        if self._h is None:
            raise ValueError("matrix was destroyed")
        if X.dim() != 2 or X.shape[0] != self.m or X.stride(1) != 1 or X.dtype != self.vector_dtype or not X.is_cuda:
            raise ValueError("X must be a CUDA (m, k) tensor of the vector type with unit column stride")
        k = X.shape[1]
        if Y is None:
            Y = torch.empty(self.n, k, dtype=self.vector_dtype, device=X.device)
        if Y.shape != (self.n, k) or Y.stride(1) != 1 or Y.dtype != self.vector_dtype:
            raise ValueError("Y must be (n, k) of the vector type with unit column stride")
        _check(load().spc5_spmm(self._h, k, X.data_ptr() if X.numel() else None, X.stride(0),
                                Y.data_ptr() if Y.numel() else None, Y.stride(0), ktile, _stream_ptr(stream)),
               "spc5_spmm")
        return Y

    def autotune(self, x: torch.Tensor, y: torch.Tensor, reps: int = 5, stream=None) -> tuple[int, float]:
        """Time the kernel variants on this matrix and keep the fastest; returns (variant, median ms)."""
        v = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(load().spc5_autotune(self._h, _ptr(x), _ptr(y), reps, ctypes.byref(v), ctypes.byref(ms),
                                    _stream_ptr(stream)), "spc5_autotune")
        return v.value, ms.value

    def set_variant(self, variant: int, stream=None):
        """Switch the short-interval kernel variant (see spc5_opts.variant)."""
        _check(load().spc5_set_variant(self._h, variant, _stream_ptr(stream)), "spc5_set_variant")
        self.variant = variant

    def launch_count(self) -> int:
        """Kernels one spmv() launches with the current variant."""
        k = ctypes.c_int()
        _check(load().spc5_launch_count(self._h, ctypes.byref(k)), "spc5_launch_count")
        return k.value

    def arrays(self) -> Arrays:
        a = Arrays()
        _check(load().spc5_export(self._h, ctypes.byref(a)), "spc5_export")
        return a

    def export(self) -> dict:
        """Host copies of the beta(r,c) arrays (via the library's copy kernel)."""
        a = self.arrays()
        vsize = {SPC5_F64: 8, SPC5_F32: 4, SPC5_BF16: 2}[self.vt]

        def fetch(ptr, nbytes, dtype, count):
            buf = torch.empty(_pad16(nbytes), dtype=torch.uint8, device="cuda")
            copy_raw(ptr, buf.data_ptr(), _pad16(nbytes))
            torch.cuda.synchronize()
            return buf.cpu().numpy()[:nbytes].view(dtype)[:count].copy()

        I = a.nintervals
        out = {
            "block_rowptr": fetch(a.block_rowptr_d, 4 * (I + 1), np.int32, I + 1),
            "block_colidx": fetch(a.block_colidx_d, 4 * a.nblocks, np.int32, a.nblocks),
            "block_masks": fetch(a.block_masks_d, a.mask_bytes * a.nblocks, np.uint8, a.mask_bytes * a.nblocks),
            "values_raw": fetch(a.values_d, vsize * a.nnz, {8: np.uint64, 4: np.uint32, 2: np.uint16}[vsize], a.nnz),
            "valptr": fetch(a.valptr_d, 8 * (I + 1), np.int64, I + 1),
            "nsegments": int(a.nsegments),
            "nblocks": int(a.nblocks),
        }
        return out

    def destroy(self):
        if self._h is not None:
            load().spc5_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def convert(rowptr: torch.Tensor, colidx: torch.Tensor, values: torch.Tensor, n: int, m: int, r: int, c: int,
            long_blocks: int = 0, seg_blocks: int = 0, variant: int = 0, order_window: int = 0,
            long_values: int = 0, stream=None) -> Matrix:
    """CSR (device tensors: int64 rowptr, int32 colidx, values) -> beta(r,c)."""
    if rowptr.dtype != torch.int64 or colidx.dtype != torch.int32:
        raise TypeError("rowptr must be int64 and colidx int32")
    if values.dtype not in _VALUE_DTYPE:
        raise TypeError("values must be float64, float32 or bfloat16")
    vt = _VALUE_DTYPE[values.dtype]
    nnz = values.numel()
    opts = Opts(long_blocks, seg_blocks, variant, order_window, long_values)
    h = ctypes.c_void_p()
    _check(load().spc5_convert(n, m, nnz, _ptr(rowptr), _ptr(colidx), _ptr(values), vt, r, c, ctypes.byref(opts),
                               _stream_ptr(stream), ctypes.byref(h)), "spc5_convert")
    M = Matrix(h.value, n, m, nnz, r, c, vt)
    M.variant = variant
    return M


def convert_rows(rowptr: torch.Tensor, colidx: torch.Tensor, values: torch.Tensor, n: int, m: int, r: int, c: int,
                 row_begin: int, row_end: int, long_blocks: int = 0, seg_blocks: int = 0, variant: int = 0,
                 order_window: int = 0, long_values: int = 0, stream=None) -> Matrix:
    """Rows [row_begin, row_end) of a device CSR -> a shard handle (full column space, rows from 0)."""
    if rowptr.dtype != torch.int64 or colidx.dtype != torch.int32:
        raise TypeError("rowptr must be int64 and colidx int32")
    vt = _VALUE_DTYPE[values.dtype]
    opts = Opts(long_blocks, seg_blocks, variant, order_window, long_values)
    h = ctypes.c_void_p()
    _check(load().spc5_convert_rows(n, m, values.numel(), _ptr(rowptr), _ptr(colidx), _ptr(values), vt, r, c,
                                    row_begin, row_end, ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(h)),
           "spc5_convert_rows")
    M = Matrix(h.value, row_end - row_begin, m, 0, r, c, vt)
    M.nnz = int(M.arrays().nnz)
    return M


def assemble(n: int, m: int, r: int, c: int, block_rowptr: torch.Tensor, block_colidx: torch.Tensor,
             block_masks: torch.Tensor, values: torch.Tensor, long_blocks: int = 0, seg_blocks: int = 0,
             variant: int = 0, order_window: int = 0, stream=None) -> Matrix:
    """beta(r,c) arrays built by the caller (device tensors: int32 block_rowptr and block_colidx,
    uint8 block_masks, values float64 / float32 / bfloat16) -> handle (arrays copied)."""
    if block_rowptr.dtype != torch.int32 or block_colidx.dtype != torch.int32 or block_masks.dtype != torch.uint8:
        raise TypeError("block_rowptr / block_colidx must be int32 and block_masks uint8")
    if values.dtype not in _VALUE_DTYPE:
        raise TypeError("values must be float64, float32 or bfloat16")
    vt = _VALUE_DTYPE[values.dtype]
    opts = Opts(long_blocks, seg_blocks, variant, order_window)
    h = ctypes.c_void_p()
    _check(load().spc5_assemble(n, m, values.numel(), block_colidx.numel(), _ptr(block_rowptr), _ptr(block_colidx),
                                _ptr(block_masks), _ptr(values), vt, r, c, ctypes.byref(opts), _stream_ptr(stream),
                                ctypes.byref(h)), "spc5_assemble")
    return Matrix(h.value, n, m, values.numel(), r, c, vt)


def csr_spmv(rowptr: torch.Tensor, colidx: torch.Tensor, values: torch.Tensor, n: int, m: int, x: torch.Tensor,
             y: torch.Tensor | None = None, group: int = 0, stream=None) -> torch.Tensor:
    """y = A x on plain CSR (the comparison kernel)."""
    vt = _VALUE_DTYPE[values.dtype]
    if y is None:
        y = torch.empty(n, dtype=_VECTOR_DTYPE[vt], device=x.device)
    _check(load().spc5_csr_spmv(n, m, values.numel(), _ptr(rowptr), _ptr(colidx), _ptr(values), vt, _ptr(x), _ptr(y),
                                group, _stream_ptr(stream)), "spc5_csr_spmv")
    return y


def tune(d: "DeviceCSR", k_spmm: int = 0, reps: int = 5, use_cache: bool = True, stream=None) -> dict:
    """Fastest (shape, variant) for the SpMV and, for k_spmm > 0, (shape, column tile) for the
    SpMM of a device CSR, timed on this GPU and remembered per matrix signature."""
    res = TuneResult()
    vt = _VALUE_DTYPE[d.values.dtype]
    _check(load().spc5_tune(d.n, d.m, d.nnz, _ptr(d.rowptr), _ptr(d.colidx), _ptr(d.values), vt, k_spmm, reps,
                            0 if use_cache else TUNE_NO_CACHE, ctypes.byref(res), _stream_ptr(stream)), "spc5_tune")
    return {f: getattr(res, f) for f, _ in TuneResult._fields_}


def pool_trim():
    """Return the memory the library keeps for reuse by later conversions."""
    _check(load().spc5_pool_trim(), "spc5_pool_trim")


class SmStream:
    """A torch stream whose kernels run on about `sms` SMs only (spc5_sm_stream_create)."""

    def __init__(self, sms: int, device=None):
        st, got = ctypes.c_void_p(), ctypes.c_int()
        _check(load().spc5_sm_stream_create(sms, ctypes.byref(st), ctypes.byref(got)), "spc5_sm_stream_create")
        self._raw, self.sms = st.value, got.value
        self.stream = torch.cuda.ExternalStream(self._raw, device=device)

    def destroy(self):
        if self._raw is not None:
            load().spc5_sm_stream_destroy(self._raw)
            self._raw = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tune_cache_clear():
    _check(load().spc5_tune_cache_clear(), "spc5_tune_cache_clear")


class CsrPlan:
    """Plain CSR with long rows split into warp segments (spc5_csr_plan_*)."""

    def __init__(self, d: "DeviceCSR", group: int = 0, long_len: int = 0, seg_len: int = 0, stream=None):
        vt = _VALUE_DTYPE[d.values.dtype]
        p = ctypes.c_void_p()
        _check(load().spc5_csr_plan_create(d.n, d.nnz, _ptr(d.rowptr), vt, group, long_len, seg_len,
                                           _stream_ptr(stream), ctypes.byref(p)), "spc5_csr_plan_create")
        self._p, self.d = p.value, d
        g, ll, ns = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().spc5_csr_plan_info(self._p, ctypes.byref(g), ctypes.byref(ll), ctypes.byref(ns)), "spc5_csr_plan_info")
        self.group, self.long_len, self.nsegments = g.value, ll.value, ns.value

    def spmv(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if y is None:
            y = torch.empty(self.d.n, dtype=x.dtype, device=x.device)
        _check(load().spc5_csr_spmv_plan(self._p, _ptr(self.d.colidx), _ptr(self.d.values), _ptr(x), _ptr(y),
                                         _stream_ptr(stream)), "spc5_csr_spmv_plan")
        return y

    def destroy(self):
        if self._p is not None:
            load().spc5_csr_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def count_blocks(rowptr: torch.Tensor, colidx: torch.Tensor, n: int, m: int, stream=None) -> np.ndarray:
    """N_blocks(r,c) for the twelve shapes (r outer, c inner), without conversion."""
    out = np.zeros(12, dtype=np.int64)
    _check(load().spc5_count_blocks(n, m, colidx.numel(), _ptr(rowptr), _ptr(colidx), out.ctypes.data,
                                    _stream_ptr(stream)), "spc5_count_blocks")
    return out


def device_peaks() -> dict:
    """Nominal DRAM GB/s, SM count and maximum SM MHz of the current device."""
    g, sms, mhz = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _check(load().spc5_device_peaks(ctypes.byref(g), ctypes.byref(sms), ctypes.byref(mhz)), "spc5_device_peaks")
    return {"hbm_gbs_nominal": g.value, "sm_count": sms.value, "sm_max_mhz": mhz.value}


def copy_raw(src_ptr: int, dst_ptr: int, nbytes: int, stream=None):
    _check(load().spc5_copy(src_ptr, dst_ptr, nbytes, _stream_ptr(stream)), "spc5_copy")


def copy(src: torch.Tensor, dst: torch.Tensor, stream=None):
    """dst = src with the library's streaming copy kernel (HBM ceiling)."""
    nbytes = src.numel() * src.element_size()
    copy_raw(_ptr(src), _ptr(dst), nbytes, stream)


def cg(A: Matrix, b: torch.Tensor, A_inner: Matrix | None = None, x: torch.Tensor | None = None, tol: float = 1e-10,
       max_iters: int = 0, max_outer: int = 0, inner_tol: float = 0.0, inner_max_iters: int = 0, check_every: int = 0,
       use_graph: bool = False, reliable: bool = False, stream=None):
    """Solve A x = b (float64 CG, or mixed precision with A_inner: refinement, or one float32
    recurrence with reliable updates when `reliable`). Returns (x, info dict)."""
    if x is None:
        x = torch.empty_like(b)
    opts = CgOpts(tol, max_iters, max_outer, inner_tol, inner_max_iters, check_every, 1 if use_graph else 0,
                  1 if reliable else 0)
    info = CgInfo()
    _check(load().spc5_cg(A._h, A_inner._h if A_inner is not None else None, _ptr(b), _ptr(x), ctypes.byref(opts),
                          ctypes.byref(info), _stream_ptr(stream)), "spc5_cg")
    return x, {"iterations": info.iterations, "outer": info.outer, "inner_total": info.inner_total,
               "converged": bool(info.converged), "rel_residual": info.rel_residual}


def features(d: "DeviceCSR", stream=None) -> np.ndarray:
    """The 16 selection features of a device CSR (no conversion)."""
    out = np.zeros(NFEATURES, dtype=np.float64)
    _check(load().spc5_features(d.n, d.m, d.nnz, _ptr(d.rowptr), _ptr(d.colidx), out.ctypes.data,
                                _stream_ptr(stream)), "spc5_features")
    return out


def time_formats(d: "DeviceCSR", reps: int = 5, stream=None) -> np.ndarray:
    """Median SpMV milliseconds for the twelve shapes (the timing recorder)."""
    vt = _VALUE_DTYPE[d.values.dtype]
    xdt = _VECTOR_DTYPE[vt]
    x = torch.rand(d.m, dtype=xdt, device=d.values.device)
    y = torch.empty(d.n, dtype=xdt, device=d.values.device)
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())  # x is written on the current stream
    out = np.zeros(NFORMATS, dtype=np.float32)
    _check(load().spc5_time_formats(d.n, d.m, d.nnz, _ptr(d.rowptr), _ptr(d.colidx), _ptr(d.values), vt, _ptr(x),
                                    _ptr(y), reps, out.ctypes.data, _stream_ptr(stream)), "spc5_time_formats")
    return out


def mlp_nparams(nfeat: int = 16) -> int:
    return int(load().spc5_mlp_nparams_n(nfeat))


def features_ext(d: "DeviceCSR", sm_frac: float = 1.0, stream=None) -> np.ndarray:
    """The 20 extended selection features (spc5_features_ext)."""
    out = np.zeros(20, dtype=np.float64)
    _check(load().spc5_features_ext(d.n, d.m, d.nnz, _ptr(d.rowptr), _ptr(d.colidx), sm_frac, out.ctypes.data,
                                    _stream_ptr(stream)), "spc5_features_ext")
    return out


def mlp_train(params: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, M: torch.Tensor, epochs: int, batch: int = 32,
              lr: float = 1e-3, seed: int = 0, stream=None) -> np.ndarray:
    """Train the format-scoring MLP (16 or 20 inputs: X.shape[1]) in place on the GPU;
    returns the per-epoch mean loss."""
    hist = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(load().spc5_mlp_train_n(_ptr(params), _ptr(X), _ptr(Y), _ptr(M), X.shape[0], X.shape[1], epochs, batch,
                                   lr, seed, hist.ctypes.data, _stream_ptr(stream)), "spc5_mlp_train")
    return hist[:epochs]


def mlp_grad(params: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, M: torch.Tensor, stream=None):
    """(loss, gradient) of the first X.shape[0] <= 32 samples."""
    g = torch.empty(mlp_nparams(X.shape[1]), dtype=torch.float32, device=params.device)
    loss = ctypes.c_float()
    _check(load().spc5_mlp_grad_n(_ptr(params), _ptr(X), _ptr(Y), _ptr(M), X.shape[0], X.shape[1],
                                  ctypes.byref(loss), _ptr(g), _stream_ptr(stream)), "spc5_mlp_grad")
    return float(loss.value), g


def mlp_infer(params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty(X.shape[0], NFORMATS, dtype=torch.float32, device=params.device)
    _check(load().spc5_mlp_infer_n(_ptr(params), _ptr(X), X.shape[0], X.shape[1], _ptr(out), _stream_ptr(stream)),
           "spc5_mlp_infer")
    return out


def partition(block_rowptr: np.ndarray, nparts: int) -> np.ndarray:
    """Interval bounds (int64[nparts + 1]) of the paper's block-balanced static partition."""
    brp = np.ascontiguousarray(block_rowptr, dtype=np.int32)
    bounds = np.zeros(nparts + 1 if nparts >= 1 else 1, dtype=np.int64)
    _check(load().spc5_partition(brp.ctypes.data, brp.shape[0] - 1, nparts, bounds.ctypes.data), "spc5_partition")
    return bounds


def poly_fit(avg: np.ndarray, perf: np.ndarray, degree: int) -> np.ndarray:
    """Per-format least-squares polynomial coefficients, shape (12, degree + 1)."""
    avg = np.ascontiguousarray(avg, dtype=np.float64)
    perf = np.ascontiguousarray(perf, dtype=np.float64)
    coef = np.zeros((NFORMATS, degree + 1), dtype=np.float64)
    _check(load().spc5_poly_fit(avg.ctypes.data, perf.ctypes.data, avg.shape[0], degree, coef.ctypes.data),
           "spc5_poly_fit")
    return coef


def poly2_fit(avg: np.ndarray, sm_frac: np.ndarray, perf: np.ndarray, degree: int) -> np.ndarray:
    """The paper's 2D regression per format over (Avg(r,c), SM fraction); (12, nterms) coefficients."""
    avg = np.ascontiguousarray(avg, dtype=np.float64)
    sf = np.ascontiguousarray(sm_frac, dtype=np.float64)
    perf = np.ascontiguousarray(perf, dtype=np.float64)
    coef = np.zeros((NFORMATS, (degree + 1) * (degree + 2) // 2), dtype=np.float64)
    _check(load().spc5_poly2_fit(avg.ctypes.data, sf.ctypes.data, perf.ctypes.data, avg.shape[0], degree,
                                 coef.ctypes.data), "spc5_poly2_fit")
    return coef


def poly2_select(coef: np.ndarray, degree: int, features: np.ndarray, sm_frac: float):
    """(r, c, estimates) of the 2D regression at one matrix and SM fraction."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    f = np.ascontiguousarray(features, dtype=np.float64)
    est = np.zeros(NFORMATS, dtype=np.float64)
    r, c = ctypes.c_int(), ctypes.c_int()
    _check(load().spc5_poly2_select(coef.ctypes.data, degree, f.ctypes.data, sm_frac, ctypes.byref(r),
                                    ctypes.byref(c), est.ctypes.data), "spc5_poly2_select")
    return r.value, c.value, est


def select(d: "DeviceCSR", method: int, poly_coef: np.ndarray | None = None, mlp_params: torch.Tensor | None = None,
           feat_mean=None, feat_scale=None, stream=None):
    """Pick (r, c) for a device CSR; returns (r, c, per-format scores)."""
    sel = Selector()
    coef = None
    if poly_coef is not None:
        coef = np.ascontiguousarray(poly_coef, dtype=np.float64)
        sel.poly_degree = coef.shape[1] - 1
        sel.poly_coef = coef.ctypes.data
    if mlp_params is not None:
        sel.mlp_params_d = _ptr(mlp_params)
    if feat_mean is not None:
        for q in range(NFEATURES):
            sel.feat_mean[q] = float(feat_mean[q])
            sel.feat_scale[q] = float(feat_scale[q])
    r, c = ctypes.c_int(), ctypes.c_int()
    score = np.zeros(NFORMATS, dtype=np.float32)
    vt = _VALUE_DTYPE[d.values.dtype]
    _check(load().spc5_select(d.n, d.m, d.nnz, _ptr(d.rowptr), _ptr(d.colidx), _ptr(d.values), vt, method,
                              ctypes.byref(sel), ctypes.byref(r), ctypes.byref(c), score.ctypes.data,
                              _stream_ptr(stream)), "spc5_select")
    return r.value, c.value, score


class Batch:
    """y_j = A_j x_j for many matrices in one persistent, graph-replayed launch."""

    def __init__(self, mats: list, xs: list, ys: list):
        n = len(mats)
        H = (ctypes.c_void_p * n)(*[m._h for m in mats])
        X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        Y = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
        b = ctypes.c_void_p()
        _check(load().spc5_batch_create(H, X, Y, n, ctypes.byref(b)), "spc5_batch_create")
        self._b = b.value
        self._keep = (list(mats), list(xs), list(ys))  # the batch refers to them

    def run(self, graph: bool = True, stream=None):
        f = load().spc5_batch_spmv if graph else load().spc5_batch_spmv_direct
        _check(f(self._b, _stream_ptr(stream)), "spc5_batch_spmv")

    def destroy(self):
        if self._b is not None:
            load().spc5_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fma_rate(dtype: torch.dtype = torch.float64, iters: int = 4096, reps: int = 5, lanes: int = 32) -> float:
    """Measured multiply-add rate of the library's probe kernel, in GFLOP/s (2 flops per FMA),
    with `lanes` active lanes per warp (counting only their FMAs)."""
    vt = {torch.float64: SPC5_F64, torch.float32: SPC5_F32}[dtype]
    sink = torch.empty(256, dtype=dtype, device="cuda")
    fmas = ctypes.c_int64()
    _check(load().spc5_fma_rate_lanes(vt, 16, lanes, _ptr(sink), ctypes.byref(fmas), _stream_ptr(None)),
           "spc5_fma_rate_lanes")
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(load().spc5_fma_rate_lanes(vt, iters, lanes, _ptr(sink), ctypes.byref(fmas), _stream_ptr(None)),
               "spc5_fma_rate_lanes")
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None or t < best else best
    return 2.0 * fmas.value / (best * 1e-3) / 1e9


@dataclass
class DeviceCSR:
    n: int
    m: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.values.numel())


def upload_csr(A, dtype: torch.dtype = torch.float64, device="cuda") -> DeviceCSR:
    """Copy a host CSR (numpy arrays) to the device, values cast to dtype."""
    rowptr = torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int64)).to(device)
    colidx = torch.from_numpy(np.ascontiguousarray(A.colidx, dtype=np.int32)).to(device)
    values = torch.from_numpy(np.ascontiguousarray(A.values, dtype=np.float64)).to(device).to(dtype)
    return DeviceCSR(A.n, A.m, rowptr, colidx, values)
