"""Seeded synthetic inputs: sparse matrices (CSR) and dense vectors.

This module only draws inputs; it holds none of the SpMV or block-format
arithmetic, so the CPU oracle and the CUDA path both take their inputs from it.
The generator is the SplitMix64 output function applied to a counter (Steele,
Lea & Flood 2014): every draw is addressed by (seed, stream, index), so the
results are independent of thread count and identical on x86-64 and aarch64.

The matrices stand in for the paper's SuiteSparse sets (Tables 1 and 2), which
are not available: stencils stand in for atmosmodd-like matrices, dense 3x3
block FEM matrices for bone010/ldoor/pwtk, R-MAT graphs for kron_g500-logn21
and uniform random rows for rajat31/ns3Da-like matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import weakref
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libspc5gen.so")

# streams of the vector generators (the matrix builders use their own)
STREAM_X = 1
STREAM_B = 2


def build(force: bool = False) -> str:
    """Compile gen.c into libspc5gen.so next to it (plain gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _GenCSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("rowptr", ctypes.POINTER(ctypes.c_int64)),
        ("colidx", ctypes.POINTER(ctypes.c_int32)),
        ("values", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_GenCSR)
        u64, i64, f64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        for name, args in {
            "gen_laplacian2d": [i64, i64],
            "gen_stencil3d": [i64, i64, i64, i32, i32, u64],
            "gen_block_fem": [i64, i32, i32, i32, f64, u64],
            "gen_rmat": [i32, i32, f64, f64, f64, i32, u64],
            "gen_uniform": [i64, i64, i32, u64],
            "gen_banded": [i64, i64, f64, u64],
            "gen_random": [i64, i64, f64, u64],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = P
        lib.gen_free.argtypes = [P]
        lib.gen_free.restype = None
        vp = ctypes.c_void_p
        lib.gen_fill_uniform.argtypes = [u64, u64, i64, f64, f64, vp]
        lib.gen_fill_normal.argtypes = [u64, u64, i64, vp]
        lib.gen_fill_dyadic.argtypes = [u64, u64, i64, i32, vp]
        lib.gen_fill_u64.argtypes = [u64, u64, i64, vp]
        lib.gen_splitmix_mix.argtypes = [u64]
        lib.gen_splitmix_mix.restype = u64
        for f in (lib.gen_fill_uniform, lib.gen_fill_normal, lib.gen_fill_dyadic, lib.gen_fill_u64):
            f.restype = None
        _lib = lib
    return _lib


@dataclass
class CSR:
    """A CSR matrix on the host: rowptr int64[n+1], colidx int32[nnz], values float64[nnz]."""

    n: int
    m: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.m))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.colidx] = self.values
        return d

    @staticmethod
    def from_dense(d: np.ndarray) -> "CSR":
        d = np.asarray(d, dtype=np.float64)
        n, m = d.shape
        rows, cols = np.nonzero(d)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rowptr, rows + 1, 1)
        return CSR(n, m, np.cumsum(rowptr), cols.astype(np.int32), d[rows, cols].copy())


def _take(ptr) -> CSR:
    if not ptr:
        raise MemoryError("generator failed (bad arguments or out of memory)")
    lib = _load()
    s = ptr.contents
    n, m, nnz = int(s.n), int(s.m), int(s.nnz)
    rowptr = np.ctypeslib.as_array(s.rowptr, shape=(n + 1,))
    colidx = np.ctypeslib.as_array(s.colidx, shape=(max(nnz, 1),))[:nnz]
    values = np.ctypeslib.as_array(s.values, shape=(max(nnz, 1),))[:nnz]
    out = CSR(n, m, rowptr, colidx, values)
    # the arrays view C memory: free it when the CSR object goes away
    weakref.finalize(out, lib.gen_free, ptr)
    return out


def laplacian2d(nx: int, ny: int) -> CSR:
    """5-point Laplacian on an nx-by-ny grid, natural ordering, values 4 / -1."""
    return _take(_load().gen_laplacian2d(nx, ny))


def stencil3d(nx: int, ny: int, nz: int, points: int = 27, normal_values: bool = True, seed: int = 1) -> CSR:
    """7- or 27-point stencil; values N(0,1) (seeded) or Poisson constants."""
    return _take(_load().gen_stencil3d(nx, ny, nz, points, 1 if normal_values else 0, seed))


def block_fem(nb: int, bs: int = 3, bmin: int = 9, bmax: int = 27, band_frac: float = 0.05, seed: int = 1) -> CSR:
    """nb block rows of bs-by-bs dense blocks, bmin..bmax blocks per block row."""
    return _take(_load().gen_block_fem(nb, bs, bmin, bmax, band_frac, seed))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         relabel: bool = True, seed: int = 1) -> CSR:
    """R-MAT graph, 2^scale vertices, edge_factor * 2^scale draws, duplicates dropped."""
    return _take(_load().gen_rmat(scale, edge_factor, a, b, c, 1 if relabel else 0, seed))


def uniform(n: int, m: int, per_row: int = 8, seed: int = 1) -> CSR:
    """Exactly per_row distinct uniform columns per row."""
    return _take(_load().gen_uniform(n, m, per_row, seed))


def banded(n: int, half_bw: int, density: float, seed: int = 1) -> CSR:
    """Random band of half-width half_bw with the given fill (diagonal always)."""
    return _take(_load().gen_banded(n, half_bw, density, seed))


def random_csr(n: int, m: int, density: float, seed: int = 1) -> CSR:
    """Small Bernoulli(density) sparse matrix for tests."""
    return _take(_load().gen_random(n, m, density, seed))


def vec_uniform(n: int, seed: int = 0, stream: int = STREAM_X, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().gen_fill_uniform(seed, stream, n, lo, hi, out.ctypes.data)
    return out


def vec_normal(n: int, seed: int = 0, stream: int = STREAM_X) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().gen_fill_normal(seed, stream, n, out.ctypes.data)
    return out


def vec_dyadic(n: int, seed: int = 0, stream: int = STREAM_X, bits: int = 20) -> np.ndarray:
    """Values k / 2^bits, k uniform in [-2^bits, 2^bits]."""
    out = np.empty(n, dtype=np.float64)
    _load().gen_fill_dyadic(seed, stream, n, bits, out.ctypes.data)
    return out


def raw_u64(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().gen_fill_u64(seed, stream, n, out.ctypes.data)
    return out


def splitmix_mix(z: int) -> int:
    return int(_load().gen_splitmix_mix(z))
