"""spc5_assemble: handles from beta(r,c) arrays built without a CSR, against
the converter and the oracle, and its checks of bad arrays."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def from_oracle(A, r, c, **kw):
    B = oracle.beta_convert(A, r, c)
    return B, spc5.assemble(A.n, A.m, r, c, dev(B.block_rowptr, torch.int32), dev(B.block_colidx, torch.int32),
                            dev(B.block_masks, torch.uint8), dev(B.values, torch.float64), **kw)


@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_assembled_equals_converted(cuda_device, r, c):
    for A in (inputs.stencil3d(9, 7, 5, points=27, seed=4), inputs.rmat(10, seed=2)):
        B, M = from_oracle(A, r, c, long_blocks=4)
        d = spc5.upload_csr(A, torch.float64, "cuda")
        N = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=4)
        ea, ec = M.export(), N.export()
        for key in ("block_rowptr", "block_colidx", "block_masks", "values_raw", "valptr"):
            assert np.array_equal(ea[key], ec[key]), key
        assert ea["nsegments"] == ec["nsegments"]
        x = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
        assert torch.equal(M.spmv(x), N.spmv(x))
        M.destroy()
        N.destroy()


def test_assembled_aligned_cover(cuda_device):
    # a cover the converter never builds: every block starts at a multiple of c
    A = inputs.random_csr(300, 257, 0.05, seed=7)
    r, c = 2, 8
    I = (A.n + r - 1) // r
    brp, cols, masks, vals = [0], [], [], []
    for it in range(I):
        rows = range(it * r, min(it * r + r, A.n))
        entries = {}
        for i, row in enumerate(rows):
            for p in range(A.rowptr[row], A.rowptr[row + 1]):
                entries.setdefault(A.colidx[p] // c, []).append((i, A.colidx[p], A.values[p]))
        for blk in sorted(entries):
            m = 0
            for i, col, _ in entries[blk]:
                m |= 1 << (i * c + col - blk * c)
            cols.append(blk * c)
            masks += [m & 0xff, m >> 8]
            vals += [v for _, _, v in sorted(entries[blk])]  # row-major inside the block
        brp.append(len(cols))
    M = spc5.assemble(A.n, A.m, r, c, dev(np.array(brp), torch.int32), dev(np.array(cols), torch.int32),
                      dev(np.array(masks), torch.uint8), dev(np.array(vals), torch.float64))
    x = inputs.vec_uniform(A.m, seed=1)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    y = M.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(np.abs(y - y_ref) <= 1e-13 * absy)
    M.destroy()


def test_assemble_rejects_bad_arrays(cuda_device):
    A = inputs.laplacian2d(6, 5)
    B = oracle.beta_convert(A, 1, 4)

    def attempt(brp=None, cols=None, masks=None, vals=None, n=A.n, m=A.m):
        brp = B.block_rowptr if brp is None else brp
        cols = B.block_colidx if cols is None else cols
        masks = B.block_masks if masks is None else masks
        vals = B.values if vals is None else vals
        try:
            spc5.assemble(n, m, 1, 4, dev(brp, torch.int32), dev(cols, torch.int32), dev(masks, torch.uint8),
                          dev(vals, torch.float64)).destroy()
        except spc5.Spc5Error as e:
            return e.status
        return spc5.OK

    assert attempt() == spc5.OK
    bad = B.block_rowptr.copy()
    bad[2], bad[3] = bad[3], bad[2] - 1
    assert attempt(brp=bad) == spc5.EINVAL  # pointer going down
    cols = B.block_colidx.copy()
    cols[1] = cols[0] + 1  # overlaps block 0 (same interval)
    assert attempt(cols=cols) == spc5.EUNSORTED
    cols = B.block_colidx.copy()
    cols[-1] = A.m  # the last block of the last row starts past the matrix
    assert attempt(cols=cols) == spc5.ERANGE
    masks = B.block_masks.copy()
    masks[-1] |= 0x8  # a bit past column m - 1 in the last block
    assert attempt(masks=masks, vals=np.append(B.values, 1.0)) == spc5.ERANGE
    assert attempt(vals=B.values[:-1]) == spc5.EINVAL  # nnz does not match the masks
