"""spc5_tune: the library's autotuner (shape x variant for the SpMV, shape x
column tile for the SpMM) and its per-signature cache."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

VALID_VARIANTS = {5, 10, 13, 15, 16, 18, 22, 23, 24, 30, 31, 32, 33}


def test_tune_choice_is_valid_correct_and_cached(cuda_device):
    spc5.tune_cache_clear()
    A = inputs.stencil3d(24, 20, 18, points=27, seed=3)
    d = spc5.upload_csr(A, torch.float64, "cuda")
    t = spc5.tune(d, reps=3)
    assert (t["r"], t["c"]) in spc5.SHAPES and t["variant"] in VALID_VARIANTS and t["spmv_ms"] > 0
    assert t["from_cache"] == 0 and t["spmm_ms"] < 0
    # the choice runs and matches the oracle
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, t["r"], t["c"], variant=t["variant"])
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    y = M.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(np.abs(y - y_ref) <= 1e-13 * absy)
    M.destroy()
    # same structure again (other values): remembered, no timing
    B = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, inputs.vec_normal(A.nnz, seed=9))
    t2 = spc5.tune(spc5.upload_csr(B, torch.float64, "cuda"), reps=3)
    assert t2["from_cache"] == 1 and t2["signature"] == t["signature"]
    assert (t2["r"], t2["c"], t2["variant"]) == (t["r"], t["c"], t["variant"])
    # forced re-timing, and another structure gets another signature
    assert spc5.tune(d, reps=3, use_cache=False)["from_cache"] == 0
    C = inputs.rmat(11, seed=2)
    t3 = spc5.tune(spc5.upload_csr(C, torch.float64, "cuda"), reps=3)
    assert t3["from_cache"] == 0 and t3["signature"] != t["signature"]
    # the value type is part of the signature
    t4 = spc5.tune(spc5.upload_csr(A, torch.float32, "cuda"), reps=3)
    assert t4["from_cache"] == 0 and t4["signature"] != t["signature"]


@pytest.mark.parametrize("k", [1, 8, 20])
def test_tune_spmm_tile(cuda_device, k):
    spc5.tune_cache_clear()
    A = inputs.uniform(2000, 1500, 9, seed=4)
    A = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, oracle.round_f32(A.values))
    d = spc5.upload_csr(A, torch.float32, "cuda")
    t = spc5.tune(d, k_spmm=k, reps=2)
    assert t["spmm_ms"] > 0 and (t["spmm_r"], t["spmm_c"]) in spc5.SHAPES
    assert t["ktile"] in ((1,) if k == 1 else (4, -8, -16, -32, 8, 16, 32)) and abs(t["ktile"]) <= 2 * k
    assert t["spmm_variant"] in VALID_VARIANTS
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, t["spmm_r"], t["spmm_c"], variant=t["spmm_variant"])
    X = oracle.round_f32(inputs.vec_uniform(A.m * k, seed=1).reshape(A.m, k))
    Y = M.spmm(torch.from_numpy(X).float().cuda(), ktile=t["ktile"]).double().cpu().numpy()
    Yref, S = oracle.csr_spmm_dot2(A, X)
    L = np.diff(A.rowptr).astype(np.float64)[:, None]
    u = 2.0**-24
    assert np.all(np.abs(Y - Yref) <= (L + 1) * u / (1 - (L + 1) * u) * S + 1e-45)
    M.destroy()


def test_tune_rejects_bad_csr(cuda_device):
    A = inputs.CSR(2, 4, np.array([0, 2, 3], np.int64), np.array([3, 1, 0], np.int32), np.ones(3))
    with pytest.raises(spc5.Spc5Error) as ei:
        spc5.tune(spc5.upload_csr(A, torch.float64, "cuda"), reps=1, use_cache=False)
    assert ei.value.status == spc5.EUNSORTED
