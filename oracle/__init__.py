"""CPU oracle for the beta(r,c) SpMV method of Bramas & Kus (2018).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may call it; the
product path never does. It shares no code with the CUDA library. Inputs come
from the seeded generators of ``paper_1801_01134_gb300.inputs`` (any object
with ``n, m, rowptr, colidx, values`` is accepted).

Each function cites the part of the paper it follows:
  * CSR SpMV (section "Sparse Matrix Vector Product (SpMV)") in plain float64
    and as a compensated Dot2 product (Ogita, Rump & Oishi 2005);
  * CSR -> beta(r,c) conversion and beta(r,c) -> CSR expansion (section
    "Block-based storage without zero padding", Eq. 1);
  * the product y += A x read straight from the beta(r,c) arrays (block
    masks decoded into (row, column, value) triples, Eq. 1);
  * the occupancy model, Eq. 1-4;
  * the static partition of section "Parallelization";
  * dense GEMV for tiny matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EUNSORTED, EDUP, ERANGE = 0, 1, 2, 3, 4

# the twelve block shapes of the GPU library: r in {1,2,4,8}, c in {4,8,16}
SHAPES = [(r, c) for r in (1, 2, 4, 8) for c in (4, 8, 16)]
# the six shapes of the paper's optimised kernels (section "Optimized kernel implementation")
PAPER_SHAPES = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


def build(force: bool = False) -> str:
    """Compile oracle.c with plain gcc (no fused contractions)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.or_csr_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.or_csr_spmv_omp.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.or_csr_spmv_dot2.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        lib.or_csr_validate.argtypes = [i64, i64, vp, vp, vp]
        lib.or_csr_validate.restype = i32
        lib.or_beta_count.argtypes = [i64, vp, vp, i32, i32, vp]
        lib.or_beta_count.restype = i64
        lib.or_beta_convert.argtypes = [i64, vp, vp, vp, i32, i32, vp, vp, vp, vp]
        lib.or_beta_convert.restype = i32
        lib.or_beta_expand.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp, vp]
        lib.or_beta_expand.restype = i32
        lib.or_beta_spmv.argtypes = [i64, i32, i32, vp, vp, vp, vp, vp, vp]
        lib.or_beta_spmv.restype = i32
        lib.or_partition.argtypes = [i64, vp, i32, vp]
        lib.or_omp_threads.restype = i32
        for f in (lib.or_csr_spmv, lib.or_csr_spmv_omp, lib.or_csr_spmv_dot2, lib.or_partition):
            f.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _csr_arrays(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    values = np.ascontiguousarray(A.values, dtype=np.float64)
    return rowptr, colidx, values


def mask_bytes(r: int, c: int) -> int:
    """Bytes of one block mask: r*c bits rounded up to whole bytes (Eq. 1)."""
    return (r * c + 7) // 8


def n_intervals(n: int, r: int) -> int:
    return (n + r - 1) // r


# ------------------------------------------------------------------ CSR SpMV

def csr_spmv(A, x: np.ndarray) -> np.ndarray:
    """Plain sequential float64 CSR SpMV, y_i = sum_j a_ij x_j."""
    rowptr, colidx, values = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    _load().or_csr_spmv(A.n, _p(rowptr), _p(colidx), _p(values), _p(x), _p(y))
    return y


def csr_spmv_omp(A, x: np.ndarray) -> np.ndarray:
    """The plain loop with rows shared among the host's OpenMP threads."""
    rowptr, colidx, values = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    _load().or_csr_spmv_omp(A.n, _p(rowptr), _p(colidx), _p(values), _p(x), _p(y))
    return y


def omp_threads() -> int:
    return int(_load().or_omp_threads())


def csr_spmv_dot2(A, x: np.ndarray):
    """Compensated SpMV (Dot2 per row). Returns (y, |A||x|)."""
    rowptr, colidx, values = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    a = np.empty(A.n, dtype=np.float64)
    _load().or_csr_spmv_dot2(A.n, _p(rowptr), _p(colidx), _p(values), _p(x), _p(y), _p(a))
    return y, a


def dense_gemv(D: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Textbook y_i = sum_j D_ij x_j with an explicit loop (tiny inputs only)."""
    n, m = D.shape
    y = np.zeros(n)
    for i in range(n):
        s = 0.0
        for j in range(m):
            s += D[i, j] * x[j]
        y[i] = s
    return y


def validate(A) -> tuple[int, int]:
    """(status, first bad row): rows sorted ascending, no repeats, in range."""
    rowptr, colidx, _ = _csr_arrays(A)
    bad = np.zeros(1, dtype=np.int64)
    st = _load().or_csr_validate(A.n, A.m, _p(rowptr), _p(colidx), _p(bad))
    return int(st), int(bad[0])


# ------------------------------------------------------------- beta(r,c)

@dataclass
class Beta:
    """The four beta(r,c) arrays of the paper plus the shape."""

    n: int
    m: int
    r: int
    c: int
    block_rowptr: np.ndarray  # int32[I+1]
    block_colidx: np.ndarray  # int32[Nb]
    block_masks: np.ndarray   # uint8[Nb*mb]
    values: np.ndarray        # float64[nnz]

    @property
    def nblocks(self) -> int:
        return int(self.block_rowptr[-1])

    @property
    def nnz(self) -> int:
        return int(self.values.shape[0])

    def avg(self) -> float:
        """Avg(r,c) = N_nnz / N_blocks(r,c)."""
        return self.nnz / self.nblocks if self.nblocks else 0.0

    def valptr(self, csr_rowptr: np.ndarray) -> np.ndarray:
        """First value of each interval: CSR rowptr[min(r*i, n)] (derived array)."""
        idx = np.minimum(np.arange(n_intervals(self.n, self.r) + 1, dtype=np.int64) * self.r, self.n)
        return np.asarray(csr_rowptr, dtype=np.int64)[idx]


def beta_count(A, r: int, c: int):
    """Blocks per interval under greedy leftmost cover; returns (counts, N_blocks)."""
    rowptr, colidx, _ = _csr_arrays(A)
    counts = np.zeros(n_intervals(A.n, r), dtype=np.int32)
    total = _load().or_beta_count(A.n, _p(rowptr), _p(colidx), r, c, _p(counts))
    return counts, int(total)


def beta_convert(A, r: int, c: int) -> Beta:
    """CSR -> beta(r,c) (greedy leftmost block starts)."""
    rowptr, colidx, values = _csr_arrays(A)
    counts, nb = beta_count(A, r, c)
    I = n_intervals(A.n, r)
    brp = np.zeros(I + 1, dtype=np.int32)
    bcol = np.zeros(max(nb, 1), dtype=np.int32)
    bmask = np.zeros(max(nb * mask_bytes(r, c), 1), dtype=np.uint8)
    bval = np.zeros(max(A.nnz, 1), dtype=np.float64)
    st = _load().or_beta_convert(A.n, _p(rowptr), _p(colidx), _p(values), r, c, _p(brp), _p(bcol), _p(bmask), _p(bval))
    if st != OK:
        raise ValueError(f"or_beta_convert failed: {st}")
    return Beta(A.n, A.m, r, c, brp, bcol[:nb].copy(), bmask[: nb * mask_bytes(r, c)].copy(), bval[: A.nnz].copy())


@dataclass
class _CSR:
    n: int
    m: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def beta_expand(B: Beta) -> _CSR:
    """beta(r,c) -> CSR by walking the blocks and their set bits in order."""
    nnz = B.nnz
    rowptr = np.zeros(B.n + 1, dtype=np.int64)
    colidx = np.zeros(max(nnz, 1), dtype=np.int32)
    values = np.zeros(max(nnz, 1), dtype=np.float64)
    brp = np.ascontiguousarray(B.block_rowptr, dtype=np.int32)
    bcol = np.ascontiguousarray(B.block_colidx if B.nblocks else np.zeros(1, np.int32), dtype=np.int32)
    bmask = np.ascontiguousarray(B.block_masks if B.nblocks else np.zeros(1, np.uint8), dtype=np.uint8)
    bval = np.ascontiguousarray(B.values if nnz else np.zeros(1), dtype=np.float64)
    st = _load().or_beta_expand(B.n, B.r, B.c, _p(brp), _p(bcol), _p(bmask), _p(bval), _p(rowptr), _p(colidx), _p(values))
    if st != OK:
        raise ValueError(f"or_beta_expand failed: {st}")
    return _CSR(B.n, B.m, rowptr, colidx[:nnz].copy(), values[:nnz].copy())


def beta_spmv(B: Beta, x: np.ndarray, y0: np.ndarray | None = None) -> np.ndarray:
    """y = y0 + A x read from the beta(r,c) arrays (y0 = 0 if omitted): every set
    mask bit is one stored value, in storage order (Eq. 1)."""
    y = np.zeros(B.n) if y0 is None else np.array(y0, dtype=np.float64, copy=True)
    x = np.ascontiguousarray(x, dtype=np.float64)
    brp = np.ascontiguousarray(B.block_rowptr, dtype=np.int32)
    bcol = np.ascontiguousarray(B.block_colidx if B.nblocks else np.zeros(1, np.int32), dtype=np.int32)
    bmask = np.ascontiguousarray(B.block_masks if B.nblocks else np.zeros(1, np.uint8), dtype=np.uint8)
    bval = np.ascontiguousarray(B.values if B.nnz else np.zeros(1), dtype=np.float64)
    st = _load().or_beta_spmv(B.n, B.r, B.c, _p(brp), _p(bcol), _p(bmask), _p(bval), _p(x), _p(y))
    if st != OK:
        raise ValueError(f"or_beta_spmv failed: {st}")
    return y


# --------------------------------------------------------- occupancy model

def occupancy_beta(n: int, nnz: int, nblocks: int, r: int, c: int, s_float: int = 8, s_int: int = 4) -> float:
    """O(r,c) of Eq. 1 in bytes, with block_rowptr counted as I+1 integers."""
    return nnz * s_float + (n_intervals(n, r) + 1) * s_int + nblocks * s_int + nblocks * r * c / 8


def occupancy_csr(n: int, nnz: int, s_float: int = 8, s_int: int = 4) -> float:
    """O_CSR of Eq. 3 (row pointer counted as n+1 integers)."""
    return nnz * s_float + (n + 1) * s_int + nnz * s_int


def break_even_avg(r: int, c: int, s_int: int = 4) -> float:
    """Eq. 4: beta(r,c) saves index bytes over CSR iff Avg(r,c) exceeds this."""
    return 1.0 + r * c / (8.0 * s_int)


# ----------------------------------------------------------- partitioning

def partition(block_rowptr: np.ndarray, nthreads: int) -> np.ndarray:
    """Interval bounds of the static block-balanced partition (section "Parallelization")."""
    brp = np.ascontiguousarray(block_rowptr, dtype=np.int32)
    bounds = np.zeros(nthreads + 1, dtype=np.int64)
    _load().or_partition(brp.shape[0] - 1, _p(brp), nthreads, _p(bounds))
    return bounds


# ------------------------------------------------------- precision forms

def round_f32(a: np.ndarray) -> np.ndarray:
    """Round float64 to the nearest float32 (ties to even), back in float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (8 significand bits, ties to even) via float32, back in float64.

    Written from the format definition: keep the top 16 bits of the float32
    pattern after adding 0x7fff plus the lowest kept bit (round half to even).
    """
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- SpMM

def csr_spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X for a dense m-by-k X, one column at a time with the plain CSR
    loop (the definition: column j of Y is the SpMV with column j of X)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.empty((A.n, X.shape[1]))
    for j in range(X.shape[1]):
        Y[:, j] = csr_spmv(A, np.ascontiguousarray(X[:, j]))
    return Y


def csr_spmm_dot2(A, X: np.ndarray):
    """Compensated Y = A X (Dot2 per entry) and |A||X| per entry."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.empty((A.n, X.shape[1]))
    S = np.empty_like(Y)
    for j in range(X.shape[1]):
        Y[:, j], S[:, j] = csr_spmv_dot2(A, np.ascontiguousarray(X[:, j]))
    return Y, S
