"""Conjugate gradients on the GPU (float64 and mixed-precision refinement)
against the CPU oracle: iteration counts, and the true residual of the
returned x recomputed by the oracle's compensated SpMV."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import cg as ocg
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu


def poisson(N):
    return inputs.stencil3d(N, N, N, points=7, normal_values=False)


def handles(A, r=2, c=4, low=torch.float32):
    d64 = spc5.upload_csr(A, torch.float64, "cuda")
    M64 = spc5.convert(d64.rowptr, d64.colidx, d64.values, A.n, A.m, r, c)
    d32 = spc5.upload_csr(A, low, "cuda")
    M32 = spc5.convert(d32.rowptr, d32.colidx, d32.values, A.n, A.m, r, c)
    return M64, M32


def true_residual(A, x, b):
    y, _ = oracle.csr_spmv_dot2(A, x)
    return np.linalg.norm(b - y) / np.linalg.norm(b)


@pytest.mark.parametrize("use_graph", [False, True])
def test_cg_f64_matches_oracle_iterations(cuda_device, use_graph):
    A = poisson(24)
    b = inputs.vec_uniform(A.n, seed=0)
    M64, _ = handles(A)
    x, info = spc5.cg(M64, torch.from_numpy(b).cuda(), tol=1e-10, check_every=1, use_graph=use_graph)
    _, k_ref, _ = ocg.cg(A, b, tol=1e-10)
    assert abs(info["iterations"] - k_ref) <= 2
    xr = x.cpu().numpy()
    assert true_residual(A, xr, b) <= 1e-10 * 1.05
    assert info["converged"] and abs(info["rel_residual"] - true_residual(A, xr, b)) <= 1e-12


def test_cg_graph_and_plain_agree_bitwise(cuda_device):
    A = poisson(20)
    b = inputs.vec_uniform(A.n, seed=3)
    M64, M32 = handles(A)
    bd = torch.from_numpy(b).cuda()
    x1, i1 = spc5.cg(M64, bd, tol=1e-10, use_graph=False)
    x2, i2 = spc5.cg(M64, bd, tol=1e-10, use_graph=True)
    assert i1["iterations"] == i2["iterations"] and torch.equal(x1, x2)
    x3, i3 = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=False)
    x4, i4 = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=True)
    assert i3 == i4 and torch.equal(x3, x4)


@pytest.mark.parametrize("low", [torch.float32, torch.bfloat16])
def test_mixed_refinement_reaches_float64_residual(cuda_device, low):
    A = poisson(24)
    b = inputs.vec_uniform(A.n, seed=0)
    M64, Ml = handles(A, low=low)  # Poisson values 6 / -1 are exact in bfloat16
    x, info = spc5.cg(M64, torch.from_numpy(b).cuda(), A_inner=Ml, tol=1e-10, inner_tol=1e-6, use_graph=True)
    xr = x.cpu().numpy()
    assert info["converged"] and true_residual(A, xr, b) <= 1e-10
    assert 1 <= info["outer"] <= 6
    _, outer_ref, inner_ref, _ = ocg.ir_cg(A, b, tol=1e-10, inner_tol=1e-6)
    assert abs(info["outer"] - outer_ref) <= 1


@pytest.mark.parametrize("low", [torch.float32, torch.bfloat16])
def test_reliable_updates_reach_float64_residual(cuda_device, low):
    A = poisson(24)
    b = inputs.vec_uniform(A.n, seed=0)
    M64, Ml = handles(A, low=low)
    bd = torch.from_numpy(b).cuda()
    x, info = spc5.cg(M64, bd, A_inner=Ml, tol=1e-10, use_graph=True, reliable=True)
    assert info["converged"] and true_residual(A, x.cpu().numpy(), b) <= 1e-10
    # one unrestarted recurrence: about the oracle's count, and no more than float64 CG's by much
    _, upd_ref, k_ref, _ = ocg.reliable_cg(A, b, tol=1e-10, delta=0.1)
    _, k64, _ = ocg.cg(A, b, tol=1e-10)
    assert abs(info["iterations"] - k_ref) <= 0.2 * k_ref + 8
    assert info["iterations"] <= 1.25 * k64 + 8
    assert info["outer"] >= 2
    # graph replay and plain launches give the same bits
    x2, info2 = spc5.cg(M64, bd, A_inner=Ml, tol=1e-10, use_graph=False, reliable=True)
    assert info2 == info and torch.equal(x, x2)


@pytest.mark.parametrize("low", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("reliable", [False, True])
def test_low_precision_cg_on_values_that_round(cuda_device, low, reliable):
    # the Poisson values 6 / -1 are exact in bfloat16, so the inner matrix of
    # the tests above equals the float64 one; with a random diagonal shift the
    # inner matrix is a rounded copy and the float64 residual has to correct it
    A = inputs.poisson_shifted(24, 24, 24, seed=4)
    rnd = oracle.round_bf16 if low == torch.bfloat16 else oracle.round_f32
    assert np.count_nonzero(rnd(A.values) != A.values) > A.n // 2
    b = inputs.vec_uniform(A.n, seed=0)
    M64, Ml = handles(A, low=low)
    x, info = spc5.cg(M64, torch.from_numpy(b).cuda(), A_inner=Ml, tol=1e-10, use_graph=True, reliable=reliable)
    assert info["converged"] and true_residual(A, x.cpu().numpy(), b) <= 1e-10
    if not reliable:
        assert info["outer"] >= 2  # at least one correction of the rounded solve


def test_cg_full_size_poisson96(cuda_device):
    # the precision-form CG workload: 7-point Poisson on a 96^3 grid, b uniform[-1,1] seed 0
    A = poisson(96)
    assert A.n == 884736 and A.nnz == 6137856
    b = inputs.vec_uniform(A.n, seed=0)
    M64, M32 = handles(A)
    lo, hi = ocg.poisson3d_eig_bounds(96, 96, 96)
    kappa = hi / lo
    bound = ocg.cg_iteration_bound(kappa, 1e-10 / math.sqrt(kappa))
    bd = torch.from_numpy(b).cuda()
    x, info = spc5.cg(M64, bd, tol=1e-10, use_graph=True)
    assert info["converged"] and info["iterations"] <= bound + 8
    assert true_residual(A, x.cpu().numpy(), b) <= 1.05e-10
    xm, im = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=True)
    assert im["converged"] and true_residual(A, xm.cpu().numpy(), b) <= 1e-10
    xr, ir = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=True, reliable=True)
    assert ir["converged"] and true_residual(A, xr.cpu().numpy(), b) <= 1e-10
    assert ir["iterations"] <= 1.15 * info["iterations"] + 8


def test_cg_with_long_interval_segments(cuda_device):
    # every interval with more than 2 blocks on the segment path: the iteration
    # then runs the SpMV and the p / q update as separate kernels
    A = poisson(16)
    b = inputs.vec_uniform(A.n, seed=5)
    d64 = spc5.upload_csr(A, torch.float64, "cuda")
    d32 = spc5.upload_csr(A, torch.float32, "cuda")
    M64 = spc5.convert(d64.rowptr, d64.colidx, d64.values, A.n, A.m, 2, 4, long_blocks=2, seg_blocks=3)
    M32 = spc5.convert(d32.rowptr, d32.colidx, d32.values, A.n, A.m, 2, 4, long_blocks=2, seg_blocks=3)
    assert M64.export()["nsegments"] > 0
    bd = torch.from_numpy(b).cuda()
    x, info = spc5.cg(M64, bd, tol=1e-10, use_graph=True)
    _, k_ref, _ = ocg.cg(A, b, tol=1e-10)
    assert info["converged"] and abs(info["iterations"] - k_ref) <= 8
    assert true_residual(A, x.cpu().numpy(), b) <= 1.05e-10
    xm, im = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=True)
    assert im["converged"] and true_residual(A, xm.cpu().numpy(), b) <= 1e-10
    xr, ir = spc5.cg(M64, bd, A_inner=M32, tol=1e-10, use_graph=True, reliable=True)
    assert ir["converged"] and true_residual(A, xr.cpu().numpy(), b) <= 1e-10
    assert ir["iterations"] <= 1.15 * info["iterations"] + 8


def test_cg_rejects_bad_handles(cuda_device):
    A = poisson(6)
    M64, M32 = handles(A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(spc5.Spc5Error):
        spc5.cg(M32, b)  # A must be float64
    with pytest.raises(spc5.Spc5Error):
        spc5.cg(M64, b, A_inner=M64)  # inner must be float32 / bfloat16
    x, info = spc5.cg(M64, torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    assert info["converged"] and torch.count_nonzero(x).item() == 0
