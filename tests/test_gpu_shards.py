"""Row shards (section "Parallelization"): the block-balanced partition of the
row intervals (spc5_partition), one handle per part (spc5_convert_rows), each
part's product written to its own rows of y. Run here on one GPU, the shards'
products must equal the whole matrix's product bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

MATS = {
    "rmat12": lambda: inputs.rmat(12, seed=4),
    "st27": lambda: inputs.stencil3d(17, 13, 11, points=27, seed=2),
    "fem": lambda: inputs.block_fem(500, seed=3),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (4, 8), (8, 16)])
@pytest.mark.parametrize("parts", [1, 3, 8])
def test_sharded_product_equals_whole(cuda_device, name, r, c, parts):
    A = MATS[name]()
    d = spc5.upload_csr(A, torch.float64, "cuda")
    x = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
    # the same long-interval thresholds in the whole matrix and every shard
    lb, lv = 48, 1024 * r
    W = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=lb, long_values=lv)
    whole = W.spmv(x)
    brp = W.export()["block_rowptr"]
    bounds = spc5.partition(brp, parts)
    assert np.array_equal(bounds, oracle.partition(brp, parts))
    y = torch.full((A.n + 16,), float("nan"), dtype=torch.float64, device="cuda")
    total_nnz = 0
    for t in range(parts):
        r0, r1 = min(int(bounds[t]) * r, A.n), min(int(bounds[t + 1]) * r, A.n)
        S = spc5.convert_rows(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, r0, r1, long_blocks=lb, long_values=lv)
        total_nnz += S.nnz
        if r1 > r0:
            S.spmv(x, y[r0:r1])
        S.destroy()
    assert total_nnz == A.nnz
    assert torch.equal(y[:A.n], whole)
    assert torch.isnan(y[A.n:]).all()
    W.destroy()


def test_shard_bounds_are_checked(cuda_device):
    A = inputs.rmat(9, seed=1)
    d = spc5.upload_csr(A, torch.float64, "cuda")
    for r0, r1, r in ((-1, 4, 1), (8, 4, 1), (0, A.n + 1, 1), (3, 8, 2)):
        with pytest.raises(spc5.Spc5Error) as ei:
            spc5.convert_rows(d.rowptr, d.colidx, d.values, A.n, A.m, r, 8, r0, r1)
        assert ei.value.status == spc5.EINVAL
