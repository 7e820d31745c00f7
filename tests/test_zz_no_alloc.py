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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_spmv_two_calls_in_a_row(cuda_device, dtype):
    A = inputs.rmat(11, seed=2)
    d = spc5.upload_csr(A, dtype, "cuda")
    # every interval with more than one block goes through the segment path,
    # so the fixed scratch array is exercised
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8, long_blocks=1, seg_blocks=3)
    assert M.export()["nsegments"] > 0
    xdt = torch.float64 if dtype == torch.float64 else torch.float32
    for seed in (0, 1):  # two calls in a row, different inputs
        xh = inputs.vec_uniform(A.m, seed=seed)
        x = torch.from_numpy(xh).to(xdt).cuda()
        y_ref = M.spmv(x)
        y = torch.full((A.n,), float("nan"), dtype=xdt, device="cuda")
        _call_noalloc(M, x, y)
        torch.cuda.synchronize()
        a, b = y.double().cpu().numpy(), y_ref.double().cpu().numpy()
        if dtype == torch.float64:
            # the test suite's float64 tolerance, against the existing entry point and the oracle
            ref, absy = oracle.csr_spmv_dot2(A, xh)
            assert np.all(np.abs(a - b) <= 1e-13 * absy)
            assert np.all(np.abs(a - ref) <= 1e-13 * absy)
        else:
            L = np.diff(A.rowptr).astype(np.float64)
            absy = oracle.csr_spmv_dot2(A, xh)[1]
            assert np.all(np.abs(a - b) <= 2 * (L + 1) * 2.0**-24 * absy + 1e-30)
    M.destroy()


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
