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
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libspc5gen.so")

# streams of the vector generators (the matrix builders use their own)
STREAM_X = 1
STREAM_B = 2
STREAM_SHIFT = 3


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
    """Copy the generator's arrays into numpy-owned memory and free the C side
    (views into C memory would dangle once their first owner is collected)."""
    if not ptr:
        raise MemoryError("generator failed (bad arguments or out of memory)")
    lib = _load()
    try:
        s = ptr.contents
        n, m, nnz = int(s.n), int(s.m), int(s.nnz)
        rowptr = np.ctypeslib.as_array(s.rowptr, shape=(n + 1,)).copy()
        colidx = np.ctypeslib.as_array(s.colidx, shape=(max(nnz, 1),))[:nnz].copy()
        values = np.ctypeslib.as_array(s.values, shape=(max(nnz, 1),))[:nnz].copy()
    finally:
        lib.gen_free(ptr)
    return CSR(n, m, rowptr, colidx, values)


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


def poisson_shifted(nx: int, ny: int, nz: int, seed: int = 4) -> CSR:
    """7-point Poisson matrix with its diagonal 6 raised by a seeded uniform
    draw in [0, 1) per row: still symmetric and strictly diagonally dominant
    (positive definite), but its diagonal values are no longer exact in
    bfloat16 or float32."""
    A = stencil3d(nx, ny, nz, points=7, normal_values=False)
    shift = vec_uniform(A.n, seed=seed, stream=STREAM_SHIFT, lo=0.0, hi=1.0)
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    on_diag = A.colidx.astype(np.int64) == rows
    vals = np.array(A.values, dtype=np.float64, copy=True)
    vals[on_diag] = vals[on_diag] + shift[rows[on_diag]]
    return CSR(A.n, A.m, A.rowptr, A.colidx, vals)


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


# ------------------------------------------------------------ timing corpus
# Matrices for the block-shape selector: families stencil 2D / 3D, banded,
# block-FEM, R-MAT and uniform in turn (index modulo 6), n log-uniform in
# [1e4, 4e6], parameters drawn from the counter generator (stream 7000 under
# the corpus seed). Training matrices are indices 0..1999 of seed 3, held-out
# ones 2000..2299.
CORPUS_FAMILIES = ("stencil2d", "stencil3d", "banded", "block_fem", "rmat", "uniform")
_STREAM_CORPUS = 7000


def corpus_params(index: int, seed: int = 3, n_min: float = 1e4, n_max: float = 4e6) -> dict:
    d = raw_u64(8, seed=seed * 1_000_003 + index, stream=_STREAM_CORPUS)
    u = (d >> np.uint64(11)).astype(np.float64) * 2.0**-53
    n = int(round(np.exp(np.log(n_min) + u[0] * (np.log(n_max) - np.log(n_min)))))
    fam = CORPUS_FAMILIES[index % len(CORPUS_FAMILIES)]
    p = {"family": fam, "index": index, "seed": seed, "n_target": n, "values_seed": int(seed * 1_000_003 + index)}
    if fam == "stencil2d":
        side = max(8, int(round(np.sqrt(n))))
        p.update(nx=side, ny=side)
    elif fam == "stencil3d":
        side = max(4, int(round(n ** (1.0 / 3.0))))
        p.update(nx=side, ny=side, nz=side, points=7 if u[1] < 0.5 else 27)
    elif fam == "banded":
        p.update(n=n, half_bw=2 + int(u[1] * 63), density=0.05 + 0.9 * u[2])
    elif fam == "block_fem":
        bs = (2, 3, 4, 6)[int(u[1] * 4)]
        bmin = 2 + int(u[2] * 11)
        p.update(nb=max(16, n // bs), bs=bs, bmin=bmin, bmax=bmin + int(u[3] * 21), band_frac=0.001 + 0.099 * u[4])
    elif fam == "rmat":
        scale = int(min(22, max(13, round(np.log2(n)))))
        a = 0.45 + 0.15 * u[1]
        bc = (1.0 - a - 0.05) / 2.0
        p.update(scale=scale, edge_factor=4 + int(u[2] * 21), a=a, b=bc, c=bc)
    else:
        p.update(n=n, per_row=2 + int(u[1] * 39))
    return p


def corpus_matrix(index: int, seed: int = 3, **kw) -> CSR:
    p = corpus_params(index, seed, **kw)
    f, vs = p["family"], p["values_seed"]
    if f == "stencil2d":
        return laplacian2d(p["nx"], p["ny"])
    if f == "stencil3d":
        return stencil3d(p["nx"], p["ny"], p["nz"], points=p["points"], normal_values=True, seed=vs)
    if f == "banded":
        return banded(p["n"], p["half_bw"], p["density"], seed=vs)
    if f == "block_fem":
        return block_fem(p["nb"], bs=p["bs"], bmin=p["bmin"], bmax=p["bmax"], band_frac=p["band_frac"], seed=vs)
    if f == "rmat":
        return rmat(p["scale"], p["edge_factor"], p["a"], p["b"], p["c"], relabel=True, seed=vs)
    return uniform(p["n"], p["n"], p["per_row"], seed=vs)


# ------------------------------------------------------------ batch corpus
# Many uneven small matrices for the batched product: n lognormal (median
# 8192, sigma 1) clipped to [1024, 65536], 3..60 entries per row; even indices
# a stencil or banded pattern, odd indices uniform random columns.
_STREAM_BATCH = 7100


def batch_matrix(index: int, seed: int = 2) -> CSR:
    d = raw_u64(6, seed=seed * 1_000_003 + index, stream=_STREAM_BATCH)
    u = (d >> np.uint64(11)).astype(np.float64) * 2.0**-53
    # standard normal from two uniforms (Box-Muller), for the lognormal size
    z = np.sqrt(-2.0 * np.log(1.0 - u[0])) * np.cos(2.0 * np.pi * u[1])
    n = int(min(65536, max(1024, round(8192.0 * np.exp(z)))))
    per_row = 3 + int(u[2] * 58)
    vs = int(seed * 1_000_003 + index)
    if index % 2 == 0:
        if u[3] < 0.5:
            side = max(2, int(round(np.sqrt(n))))
            return laplacian2d(side, max(1, n // side)) if per_row < 8 else \
                stencil3d(max(2, round(n ** (1 / 3))), max(2, round(n ** (1 / 3))), max(2, round(n ** (1 / 3))),
                          points=27 if per_row > 16 else 7, normal_values=True, seed=vs)
        return banded(n, max(1, per_row // 2), min(0.95, per_row / (2.0 * max(1, per_row // 2) + 1)), seed=vs)
    return uniform(n, n, per_row, seed=vs)
