"""Multi-RHS SpMM (Y = A X) against the oracle, column by column."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

MATS = {
    "st27_ragged": lambda: inputs.stencil3d(13, 11, 7, points=27, seed=4),
    "rmat11": lambda: inputs.rmat(11, seed=2),
    "uniform": lambda: inputs.uniform(3001, 2500, 8, seed=5),
    "fem": lambda: inputs.block_fem(500, seed=6),
}
_cache = {}


def get(name):
    if name not in _cache:
        _cache[name] = MATS[name]()
    return _cache[name]


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (4, 16), (8, 8)])
@pytest.mark.parametrize("k,ktile", [(1, 0), (3, 4), (8, 0), (13, 8), (32, 0), (32, 32), (5, 1), (13, -8), (20, -16)])
def test_spmm_f64(cuda_device, name, r, c, k, ktile):
    A = get(name)
    X = inputs.vec_uniform(A.m * k, seed=k).reshape(A.m, k)
    Yref, S = oracle.csr_spmm_dot2(A, X)
    d = spc5.upload_csr(A, torch.float64, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=4 if name == "rmat11" else 0)
    # padded leading dimensions; NaN guard columns must stay untouched
    ld = k + 3
    Xd = torch.zeros(A.m, ld, dtype=torch.float64, device="cuda")
    Xd[:, :k] = torch.from_numpy(X)
    Yd = torch.full((A.n, ld), float("nan"), dtype=torch.float64, device="cuda")
    M.spmm(Xd[:, :k], Yd[:, :k], ktile=ktile)
    Y = Yd.cpu().numpy()
    assert np.all(np.abs(Y[:, :k] - Yref) <= 1e-13 * S), np.abs(Y[:, :k] - Yref).max()
    assert np.isnan(Y[:, k:]).all()
    M.destroy()


@pytest.mark.parametrize("name", ["st27_ragged", "rmat11"])
@pytest.mark.parametrize("k", [4, 16, 32])
def test_spmm_f32_and_column_equals_spmv(cuda_device, name, k):
    A = get(name)
    Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, oracle.round_f32(A.values))
    X = oracle.round_f32(inputs.vec_uniform(A.m * k, seed=k)).reshape(A.m, k)
    Yref, S = oracle.csr_spmm_dot2(Ar, X)
    d = spc5.upload_csr(Ar, torch.float32, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 8)
    Xd = torch.from_numpy(X).float().cuda()
    Y = M.spmm(Xd).double().cpu().numpy()
    L = np.diff(A.rowptr).astype(np.float64)[:, None]
    u = 2.0**-24
    assert np.all(np.abs(Y - Yref) <= (L + 1) * u / (1 - (L + 1) * u) * S + 1e-45)
    # column j of Y is the SpMV with column j of X
    for j in (0, k - 1):
        yj = M.spmv(Xd[:, j].contiguous()).double().cpu().numpy()
        assert np.all(np.abs(Y[:, j] - yj) <= 2 * (L[:, 0] + 1) * u * S[:, j] + 1e-45)
    M.destroy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ktile", [4, -8, -16, -32])
@pytest.mark.parametrize("pad", [0, 1])
def test_spmm_row_tiles_vector_and_scalar_loads(cuda_device, dtype, ktile, pad):
    # pad 0: X rows 16-byte aligned (vector loads of X); pad 1: scalar loads; k not a
    # multiple of the tile, so the last tile is partial either way
    A = get("st27_ragged")
    k = 2 * abs(ktile) + 3
    vals = A.values if dtype == torch.float64 else oracle.round_f32(A.values)
    Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, vals)
    X = inputs.vec_uniform(A.m * k, seed=7).reshape(A.m, k)
    if dtype == torch.float32:
        X = oracle.round_f32(X)
    Yref, S = oracle.csr_spmm_dot2(Ar, X)
    d = spc5.upload_csr(Ar, dtype, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 8)
    ld = k + pad if pad else ((k + 3) // 4) * 4
    Xd = torch.zeros(A.m, ld, dtype=dtype, device="cuda")
    Xd[:, :k] = torch.from_numpy(X).to(dtype)
    Y = M.spmm(Xd[:, :k], ktile=ktile).double().cpu().numpy()
    L = np.diff(A.rowptr).astype(np.float64)[:, None]
    if dtype == torch.float64:
        assert np.all(np.abs(Y - Yref) <= 1e-13 * S)
    else:
        u = 2.0**-24
        assert np.all(np.abs(Y - Yref) <= (L + 1) * u / (1 - (L + 1) * u) * S + 1e-45)
    M.destroy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("k", [8, 17, 32, 45])
@pytest.mark.parametrize("pad", [0, 1])
@pytest.mark.parametrize("ktile", [0, -32, 16])
def test_spmm_long_rows_column_groups(cuda_device, dtype, k, pad, ktile):
    # beta(1,c) long intervals with k >= 8 go to the column-group segment
    # kernel (2, 4 or 8 lanes of 4 columns per stored value); most R-MAT rows
    # are long here (long_blocks 2); aligned X rows (pad 0: 16-byte loads) and
    # unaligned ones (pad 1: scalar loads), partial last tiles
    A = get("rmat11")
    vals = A.values if dtype == torch.float64 else (oracle.round_f32(A.values) if dtype == torch.float32
                                                    else oracle.round_bf16(A.values))
    Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, vals)
    X = inputs.vec_uniform(A.m * k, seed=3).reshape(A.m, k)
    xdt = torch.float64 if dtype == torch.float64 else torch.float32
    if xdt == torch.float32:
        X = oracle.round_f32(X)
    Yref, S = oracle.csr_spmm_dot2(Ar, X)
    d = spc5.upload_csr(Ar, dtype, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 4, long_blocks=2)
    assert M.arrays().nsegments > 0
    ld = k + pad if pad else ((k + 3) // 4) * 4
    Xd = torch.zeros(A.m, ld, dtype=xdt, device="cuda")
    Xd[:, :k] = torch.from_numpy(X).to(xdt)
    Yd = torch.full((A.n, ld), float("nan"), dtype=xdt, device="cuda")
    M.spmm(Xd[:, :k], Yd[:, :k], ktile=ktile)
    Y = Yd.double().cpu().numpy()
    if dtype == torch.float64:
        assert np.all(np.abs(Y[:, :k] - Yref) <= 1e-13 * S)
    else:
        L = np.diff(A.rowptr).astype(np.float64)[:, None]
        u = 2.0**-24
        assert np.all(np.abs(Y[:, :k] - Yref) <= (L + 1) * u / (1 - (L + 1) * u) * S + 1e-45)
    if ld > k:
        assert np.isnan(Y[:, k:]).all()
    # repeated products give the same bits
    Y2 = torch.full_like(Yd, float("nan"))
    M.spmm(Xd[:, :k], Y2[:, :k], ktile=ktile)
    assert torch.equal(Y2[:, :k], Yd[:, :k])
    M.destroy()


def test_spmm_rejects_bad_arguments(cuda_device):
    A = get("uniform")
    d = spc5.upload_csr(A, torch.float32, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8)
    X = torch.zeros(A.m, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(spc5.Spc5Error):
        M.spmm(X, ktile=3)
    with pytest.raises(ValueError):
        M.spmm(X.double())
    M.destroy()
