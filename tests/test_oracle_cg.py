"""Pins of the CG / iterative-refinement oracle against textbook facts."""
import math

import numpy as np

import oracle
from oracle import cg as ocg
from paper_1801_01134_gb300 import inputs


def spd_random(n, seed):
    rng = np.random.default_rng(seed)
    B = (rng.random((n, n)) < 0.1) * rng.standard_normal((n, n))
    D = B @ B.T + n * np.eye(n)
    return D


def test_cg_matches_lapack_on_small_spd():
    for seed in range(4):
        D = spd_random(60, seed)
        A = inputs.CSR.from_dense(D)
        b = inputs.vec_uniform(60, seed=seed)
        x, k, hist = ocg.cg(A, b, tol=1e-13)
        ref = np.linalg.solve(D, b)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
        assert hist[-1] <= 1e-13


def test_cg_finite_termination_distinct_eigenvalues():
    # in exact arithmetic CG ends after as many steps as A has distinct eigenvalues
    d = np.array([1.0, 4.0, 9.0] * 40)
    A = inputs.CSR.from_dense(np.diag(d))
    b = inputs.vec_uniform(120, seed=1)
    x, k, hist = ocg.cg(A, b, tol=1e-12)
    assert k <= 4
    assert np.allclose(x, b / d, rtol=1e-12, atol=0)


def test_poisson_eigenvalues_closed_form_small():
    N = 5
    A = inputs.stencil3d(N, N, N, points=7, normal_values=False)
    ev = np.linalg.eigvalsh(A.to_dense())
    lo, hi = ocg.poisson3d_eig_bounds(N, N, N)
    assert abs(ev[0] - lo) < 1e-12 and abs(ev[-1] - hi) < 1e-12


def test_cg_iterations_within_classical_bound():
    N = 20
    A = inputs.stencil3d(N, N, N, points=7, normal_values=False)
    b = inputs.vec_uniform(A.n, seed=0)
    lo, hi = ocg.poisson3d_eig_bounds(N, N, N)
    kappa = hi / lo
    x, k, hist = ocg.cg(A, b, tol=1e-10)
    # ||r_k|| / ||b|| <= sqrt(kappa) ||e_k||_A / ||e_0||_A  (x0 = 0)
    bound = ocg.cg_iteration_bound(kappa, 1e-10 / math.sqrt(kappa))
    assert hist[-1] <= 1e-10 and k <= bound
    # the residual the loop reports is the true one (no drift beyond rounding)
    true = np.linalg.norm(b - oracle.csr_spmv(A, x)) / np.linalg.norm(b)
    assert true <= 2e-10


def test_ir_cg_reaches_float64_accuracy():
    N = 16
    A = inputs.stencil3d(N, N, N, points=7, normal_values=False)
    b = inputs.vec_uniform(A.n, seed=0)
    x, outer, inner, hist = ocg.ir_cg(A, b, tol=1e-10, inner_tol=1e-4)
    true = np.linalg.norm(b - oracle.csr_spmv(A, x)) / np.linalg.norm(b)
    assert true <= 1e-10 and hist[-1] == true
    # each refinement step gains about the inner tolerance
    assert outer <= 5
    x64, k64, _ = ocg.cg(A, b, tol=1e-10)
    assert np.linalg.norm(x - x64) <= 1e-8 * np.linalg.norm(x64)


def test_reliable_cg_reaches_float64_accuracy_with_cg_iteration_count():
    # the float32 recurrence is never restarted, so it needs about as many
    # iterations as float64 CG (refinement with restarts needs more), and the
    # returned x solves the system to the float64 tolerance (checked against
    # a direct solve)
    A = inputs.stencil3d(12, 12, 12, points=7, normal_values=False)
    b = inputs.vec_uniform(A.n, seed=0)
    _, k64, _ = ocg.cg(A, b, tol=1e-10)
    x, updates, k, hist = ocg.reliable_cg(A, b, tol=1e-10, delta=0.1)
    assert hist[-1] <= 1e-10 and updates >= 2
    assert k <= 1.15 * k64 + 5
    _, _, inner_ir, _ = ocg.ir_cg(A, b, tol=1e-10, inner_tol=1e-6)
    assert k <= inner_ir
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_reliable_cg_zero_rhs():
    A = inputs.stencil3d(4, 4, 4, points=7, normal_values=False)
    x, updates, k, hist = ocg.reliable_cg(A, np.zeros(A.n))
    assert updates == 0 and k == 0 and not x.any()
