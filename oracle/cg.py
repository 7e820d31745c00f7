"""CPU oracle for conjugate gradients (CG) and mixed-precision iterative
refinement around it.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). The paper names CG as the
typical consumer of many SpMVs with one matrix (Introduction); the method
here is textbook:
  * CG of Hestenes & Stiefel (1952) in float64, starting from x = 0;
  * iterative refinement (Wilkinson; Moler 1967): the residual r = b - A x,
    the update x += d and all norms in float64, the correction d solved
    approximately by CG in float32 on the float32-rounded matrix;
  * CG in float32 with reliable updates (Sleijpen & van der Vorst 1996): the
    float64 residual replaces the recurred one from time to time instead of
    restarting the iteration.
"""
from __future__ import annotations

import math

import numpy as np

from . import csr_spmv


def _spmv32(A, vals32: np.ndarray, x32: np.ndarray) -> np.ndarray:
    """float32 SpMV: float32 products, float32 sums per row (row order)."""
    prod = (vals32 * x32[A.colidx]).astype(np.float32)
    out = np.zeros(A.n, dtype=np.float32)
    starts = A.rowptr[:-1]
    nonempty = np.diff(A.rowptr) > 0
    if prod.size:
        sums = np.add.reduceat(prod, starts[nonempty]).astype(np.float32)
        out[nonempty] = sums
    return out


def cg(A, b: np.ndarray, tol: float = 1e-10, maxit: int = 100000, x0: np.ndarray | None = None):
    """float64 CG (Hestenes-Stiefel). Stops when ||r||_2 <= tol ||b||_2.

    Returns (x, iterations, history of ||r|| / ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - csr_spmv(A, x)
    p = r.copy()
    rho = float(r @ r)
    bn = math.sqrt(float(b @ b))
    hist = [math.sqrt(rho) / bn if bn else 0.0]
    k = 0
    while hist[-1] > tol and k < maxit:
        q = csr_spmv(A, p)
        pq = float(p @ q)
        if pq == 0.0:
            break
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        rho_new = float(r @ r)
        beta = rho_new / rho
        p = r + beta * p
        rho = rho_new
        k += 1
        hist.append(math.sqrt(rho) / bn)
    return x, k, hist


def cg32(A, vals32: np.ndarray, b32: np.ndarray, tol: float, maxit: int):
    """CG with float32 vectors and matrix values (inner solver of the refinement)."""
    x = np.zeros_like(b32)
    r = b32.copy()
    p = r.copy()
    rho = np.float32(r @ r)
    bn = math.sqrt(float(rho))
    k = 0
    while k < maxit and math.sqrt(float(rho)) > tol * bn:
        q = _spmv32(A, vals32, p)
        pq = np.float32(p @ q)
        if pq == 0:
            break
        alpha = np.float32(rho / pq)
        x = (x + alpha * p).astype(np.float32)
        r = (r - alpha * q).astype(np.float32)
        rho_new = np.float32(r @ r)
        beta = np.float32(rho_new / rho)
        p = (r + beta * p).astype(np.float32)
        rho = rho_new
        k += 1
    return x, k


def ir_cg(A, b: np.ndarray, tol: float = 1e-10, inner_tol: float = 1e-5, inner_maxit: int = 1000,
          max_outer: int = 50, vals_low: np.ndarray | None = None):
    """Iterative refinement: float64 residual / update / norms, float32 inner CG.

    vals_low: the matrix values the inner solver uses (float32-rounded by default).
    Returns (x, outer steps, total inner iterations, history of ||r|| / ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    vals32 = (np.asarray(A.values, dtype=np.float64) if vals_low is None else vals_low).astype(np.float32)
    x = np.zeros_like(b)
    r = b.copy()
    bn = math.sqrt(float(b @ b))
    hist = [math.sqrt(float(r @ r)) / bn if bn else 0.0]
    outer = inner = 0
    while hist[-1] > tol and outer < max_outer:
        rn = math.sqrt(float(r @ r))
        d32, k = cg32(A, vals32, (r / rn).astype(np.float32), inner_tol, inner_maxit)
        x += rn * d32.astype(np.float64)
        r = b - csr_spmv(A, x)
        outer += 1
        inner += k
        hist.append(math.sqrt(float(r @ r)) / bn)
    return x, outer, inner, hist


def reliable_cg(A, b: np.ndarray, tol: float = 1e-10, delta: float = 0.1, maxit: int = 100000,
                vals_low: np.ndarray | None = None):
    """Mixed-precision CG with reliable updates (Sleijpen & van der Vorst, 1996):
    one CG recurrence in float32 on the float32 matrix, never restarted;
    whenever the recurred residual norm has fallen below delta times its value
    at the last update (or below tol ||b|| / 2), the float32 iterate is added
    to the float64 solution (and reset), the residual b - A x is recomputed in
    float64 and replaces the recurred one, and the search direction is kept
    (beta uses the replaced residual's norm).

    Returns (x, reliable updates, float32 iterations, history of the true
    ||r|| / ||b|| at the updates)."""
    b = np.asarray(b, dtype=np.float64)
    vals32 = (np.asarray(A.values, dtype=np.float64) if vals_low is None else vals_low).astype(np.float32)
    bn = math.sqrt(float(b @ b))
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0, [0.0]
    r = b.astype(np.float32)
    x32 = np.zeros_like(r)
    p = r.copy()
    rho = np.float32(r @ r)
    rn_upd = math.sqrt(float(rho))
    hist = [1.0]
    k = updates = 0
    while k < maxit:
        q = _spmv32(A, vals32, p)
        pq = np.float32(p @ q)
        if pq == 0:
            break
        alpha = np.float32(rho / pq)
        x32 = (x32 + alpha * p).astype(np.float32)
        r = (r - alpha * q).astype(np.float32)
        rho_new = np.float32(r @ r)
        k += 1
        if math.sqrt(float(rho_new)) <= max(delta * rn_upd, 0.5 * tol * bn):
            x += x32.astype(np.float64)
            x32[:] = 0
            r64 = b - csr_spmv(A, x)
            updates += 1
            rn = math.sqrt(float(r64 @ r64))
            hist.append(rn / bn)
            if rn <= tol * bn:
                break
            r = r64.astype(np.float32)
            rho_new = np.float32(r @ r)
            rn_upd = rn
        beta = np.float32(rho_new / rho)
        p = (r + beta * p).astype(np.float32)
        rho = rho_new
    return x, updates, k, hist


def poisson3d_eig_bounds(nx: int, ny: int, nz: int) -> tuple[float, float]:
    """Extreme eigenvalues of the 7-point Dirichlet Laplacian (diagonal 6,
    off-diagonals -1): lambda = sum_d (2 - 2 cos(pi j_d / (N_d + 1)))."""
    lo = sum(2 - 2 * math.cos(math.pi / (N + 1)) for N in (nx, ny, nz))
    hi = sum(2 - 2 * math.cos(math.pi * N / (N + 1)) for N in (nx, ny, nz))
    return lo, hi


def cg_iteration_bound(kappa: float, eps: float) -> float:
    """Classical CG bound: ||e_k||_A <= 2 ((sqrt k - 1)/(sqrt k + 1))^k ||e_0||_A,
    so k >= sqrt(kappa)/2 ln(2/eps) iterations reduce the A-norm error by eps."""
    return 0.5 * math.sqrt(kappa) * math.log(2.0 / eps)
