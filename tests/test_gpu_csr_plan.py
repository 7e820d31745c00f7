"""The CSR comparator with long rows split into warp segments (the β path's
load balancing) against the compensated oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

MATS = {"rmat12": lambda: inputs.rmat(12, seed=4), "fem": lambda: inputs.block_fem(400, seed=3),
        "sparse": lambda: inputs.random_csr(203, 90, 0.004, seed=9), "uniform": lambda: inputs.uniform(3001, 2500, 8, seed=5)}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("group", [0, 1, 4, 32])
@pytest.mark.parametrize("long_len,seg_len", [(0, 0), (20, 7), (3, 2)])
def test_csr_plan_against_oracle(cuda_device, name, group, long_len, seg_len):
    A = MATS[name]()
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = spc5.upload_csr(A, torch.float64, "cuda")
    P = spc5.CsrPlan(d, group=group, long_len=long_len, seg_len=seg_len)
    if long_len == 3 and np.diff(A.rowptr).max() > 3:
        assert P.nsegments > 0
    xd = torch.from_numpy(x).cuda()
    buf = torch.full((A.n + 16,), float("nan"), dtype=torch.float64, device="cuda")
    P.spmv(xd, buf[:A.n])
    y = buf[:A.n].cpu().numpy()
    assert np.all(np.abs(y - y_ref) <= 1e-13 * absy)
    assert np.all(y[absy == 0] == 0)
    assert torch.isnan(buf[A.n:]).all()
    assert torch.equal(P.spmv(xd), buf[:A.n])  # a fixed order
    P.destroy()
    # float32 and bfloat16 values, float32 accumulation
    L = np.diff(A.rowptr).astype(np.float64)
    u = 2.0**-24
    xr = oracle.round_f32(x)
    for vdt, rnd in ((torch.float32, oracle.round_f32), (torch.bfloat16, oracle.round_bf16)):
        Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, rnd(A.values))
        yr, ar = oracle.csr_spmv_dot2(Ar, xr)
        dr = spc5.upload_csr(Ar, vdt, "cuda")
        P = spc5.CsrPlan(dr, group=group, long_len=long_len, seg_len=seg_len)
        y = P.spmv(torch.from_numpy(xr).float().cuda()).double().cpu().numpy()
        assert np.all(np.abs(y - yr) <= (L + 1) * u / (1 - (L + 1) * u) * ar + 1e-45)
        P.destroy()
