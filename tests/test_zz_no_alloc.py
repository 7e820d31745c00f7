"""spc5_spmv_noalloc: the entry point for callers that cannot let the library
allocate device memory (memory owned by another component's pool, or a fixed
budget). It keeps its segment scratch in a fixed array inside the library, so
its results must equal those of spc5_spmv, call after call, although the
array is shared and keeps the previous call's contents.

This file is collected last on purpose, so that a stop-at-first-failure run
has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu


def _call_noalloc(M, x, y):
    lib = spc5.load()
    st = lib.spc5_spmv_noalloc(ctypes.c_void_p(M._h), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == spc5.OK, spc5.last_error()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_noalloc_matches_spmv_two_calls_in_a_row(cuda_device, dtype):
    # two matrices whose segment scratch differs in size and layout (8 rows per
    # interval, then 1), called alternately: whatever one call leaves in the
    # shared array must not show in the next. The kernels are those of
    # spc5_spmv with only the scratch address changed, so the results must be
    # the same bits.
    A = inputs.rmat(11, seed=2)
    B = inputs.stencil3d(9, 8, 7, points=27, seed=3)
    da = spc5.upload_csr(A, dtype, "cuda")
    db = spc5.upload_csr(B, dtype, "cuda")
    # every interval with more than one block goes through the segment path
    Ma = spc5.convert(da.rowptr, da.colidx, da.values, A.n, A.m, 8, 4, long_blocks=1, seg_blocks=2)
    Mb = spc5.convert(db.rowptr, db.colidx, db.values, B.n, B.m, 1, 8, long_blocks=1, seg_blocks=1)
    na, nb = Ma.export()["nsegments"], Mb.export()["nsegments"]
    assert na > 0 and nb > 0 and na * 8 != nb
    xdt = torch.float64 if dtype == torch.float64 else torch.float32
    for seed in (0, 1):  # two calls in a row per matrix, different inputs
        for M, Acsr in ((Ma, A), (Mb, B)):
            xh = inputs.vec_uniform(Acsr.m, seed=seed)
            x = torch.from_numpy(xh).to(xdt).cuda()
            y_ref = M.spmv(x)
            y = torch.full((Acsr.n,), float("nan"), dtype=xdt, device="cuda")
            _call_noalloc(M, x, y)
            torch.cuda.synchronize()
            assert torch.equal(y, y_ref)
            if dtype == torch.float64:
                ref, absy = oracle.csr_spmv_dot2(Acsr, xh)
                assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-13 * absy)
    Ma.destroy()
    Mb.destroy()


def test_noalloc_rejects_oversized_scratch(cuda_device):
    # 8-row intervals split into one-block segments: 2^19 segments x 8 rows x 8 bytes > 4 MiB
    n = 1 << 19
    rowptr = np.arange(n + 1, dtype=np.int64) * 2
    colidx = np.stack([np.zeros(n, np.int64), np.full(n, 100, np.int64)], axis=1).reshape(-1).astype(np.int32)
    A = inputs.CSR(n, 200, rowptr, colidx, np.ones(2 * n))
    d = spc5.upload_csr(A, torch.float64, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, n, 200, 8, 4, long_blocks=1, seg_blocks=1)
    need = M.export()["nsegments"] * 8 * 8
    assert need > 4 << 20
    x = torch.ones(200, dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(spc5.Spc5Error) as ei:
        M.spmv_noalloc(x, y)
    assert ei.value.status == spc5.ERANGE
    M.destroy()
