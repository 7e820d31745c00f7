"""Batched product of many uneven matrices (one graph-replayed persistent
launch) against one SpMV per matrix and against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu


def build(count, dtype, seed=2):
    mats, hs, xs, ys, As = [], [], [], [], []
    xdt = torch.float64 if dtype == torch.float64 else torch.float32
    for j in range(count):
        A = inputs.batch_matrix(j, seed=seed)
        if dtype != torch.float64:
            A = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, oracle.round_f32(A.values))
        r, c = spc5.SHAPES[j % 12]
        d = spc5.upload_csr(A, dtype, "cuda")
        # every fifth matrix sends its longer intervals down the segment path
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=2 if j % 5 == 0 else 0)
        x = torch.from_numpy(inputs.vec_uniform(A.m, seed=j)).to(xdt).cuda()
        y = torch.full((A.n,), float("nan"), dtype=xdt, device="cuda")
        mats.append(M)
        hs.append(d)
        xs.append(x)
        ys.append(y)
        As.append(A)
    return As, mats, hs, xs, ys


@pytest.mark.parametrize("graph", [True, False])
def test_batch_f32_matches_single_products_bitwise(cuda_device, graph):
    As, mats, hs, xs, ys = build(40, torch.float32)
    assert any(M.export()["nsegments"] > 0 for M in mats)
    B = spc5.Batch(mats, xs, ys)
    for rnd in range(2):  # replay with new x contents
        if rnd == 1:
            for j, x in enumerate(xs):
                x.copy_(torch.from_numpy(inputs.vec_uniform(x.numel(), seed=100 + j)).float())
        B.run(graph=graph)
        torch.cuda.synchronize()
        for j, (A, M) in enumerate(zip(As, mats)):
            single = M.spmv(xs[j])
            assert torch.equal(ys[j], single), j
            xh = xs[j].double().cpu().numpy()
            yref, absy = oracle.csr_spmv_dot2(A, xh)
            L = np.diff(A.rowptr).astype(np.float64)
            u = 2.0**-24
            assert np.all(np.abs(ys[j].double().cpu().numpy() - yref) <= (L + 1) * u / (1 - (L + 1) * u) * absy + 1e-45)
    B.destroy()


def test_batch_f64_against_oracle(cuda_device):
    As, mats, hs, xs, ys = build(12, torch.float64, seed=5)
    B = spc5.Batch(mats, xs, ys)
    B.run()
    torch.cuda.synchronize()
    for j, A in enumerate(As):
        yref, absy = oracle.csr_spmv_dot2(A, xs[j].cpu().numpy())
        assert np.all(np.abs(ys[j].cpu().numpy() - yref) <= 1e-13 * absy)
    B.destroy()


def test_batch_rejects_mixed_types(cuda_device):
    A = inputs.batch_matrix(1)
    d64 = spc5.upload_csr(A, torch.float64, "cuda")
    d32 = spc5.upload_csr(A, torch.float32, "cuda")
    M64 = spc5.convert(d64.rowptr, d64.colidx, d64.values, A.n, A.m, 2, 4)
    M32 = spc5.convert(d32.rowptr, d32.colidx, d32.values, A.n, A.m, 2, 4)
    x64 = torch.zeros(A.m, dtype=torch.float64, device="cuda")
    x32 = torch.zeros(A.m, dtype=torch.float32, device="cuda")
    with pytest.raises(spc5.Spc5Error):
        spc5.Batch([M64, M32], [x64, x32], [torch.empty_like(x64), torch.empty_like(x32)])


def test_batch_keeps_each_matrix_decode_bitwise(cuda_device):
    # per-matrix tuned variants: the batch groups the matrices by shape and
    # decode and runs each with its mask-window, single-value, unrolled or
    # flattened decode, which add in storage order like the single product
    As, mats, hs, xs, ys = build(36, torch.float32, seed=7)
    for j, M in enumerate(mats):
        choices = (13, 15, 30, 31, 12, 5, 16, 18) if M.r == 1 else (12, 13, 15, 5)
        M.set_variant(choices[j % len(choices)])
    B = spc5.Batch(mats, xs, ys)
    B.run()
    torch.cuda.synchronize()
    for j, M in enumerate(mats):
        assert torch.equal(ys[j], M.spmv(xs[j])), (j, M.r, M.c)
    B.destroy()
