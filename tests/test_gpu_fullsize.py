"""Parity at the benchmarked sizes: the four matrices the bench times, at full size.

The small parity tests never reach several paths that only large inputs take:
the multi-step scan of the tile sums (more than 4096 tiles of 2048 counts, e.g.
the r = 1 block numbering over the 162 M entries of the FEM matrix), the
fix-up's warp path for long intervals of more than 32 segments (R-MAT hubs of
~10^5 entries), and the segment + short-interval grid at hundreds of thousands
of segments. Here every conversion is compared with the oracle bit for bit,
float64 products with the compensated oracle within 1e-13 (|A||x|)_i, and the
float32 / bfloat16 storage forms with an oracle fed the same rounded values
within gamma_{L_i+1} (|A||x|)_i (u = 2^-24, L_i = row length), for the block
shapes and kernel variants the bench selects and the default variant.

Matrices (section "Test matrices" stand-ins; values N(0,1) seed 1, x uniform
[-1,1] seed 0): 27-point stencil 128^3, 3x3-block FEM n = 3e6, R-MAT scale 22,
uniform n = 1e6 with 8 entries per row.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

TOL64 = 1e-13
U32 = 2.0**-24

# (r, c, variant) per matrix and value type: the bench's tuned choices, the
# default decode and a second shape
CASES = {
    "stencil27_128^3": {"f64": [(4, 8, 5), (4, 8, 15), (2, 4, 5), (4, 8, 25)],
                        "f32": [(1, 4, 18), (2, 4, 18), (4, 8, 16), (1, 4, 25), (1, 4, 32)],
                        "bf16": [(1, 4, 16), (2, 4, 18), (4, 8, 5), (1, 4, 24)]},
    "fem3x3_n3M": {"f64": [(1, 8, 22), (1, 4, 23), (1, 8, 5), (4, 4, 5), (1, 4, 25)],
                   "f32": [(1, 4, 32), (1, 4, 16), (1, 8, 22), (1, 4, 25), (1, 8, 32)],
                   "bf16": [(1, 4, 32), (1, 8, 22), (2, 8, 18), (1, 4, 26)]},
    "rmat_s22": {"f64": [(1, 4, 30), (1, 4, 15), (1, 4, 5), (1, 8, 13), (1, 4, 29)],
                 "f32": [(1, 4, 30), (1, 4, 15), (1, 8, 22), (1, 4, 28), (1, 4, 32)],
                 "bf16": [(1, 4, 30), (1, 4, 15), (1, 4, 29)]},
    "uniform_n1M": {"f64": [(1, 4, 22), (1, 4, 5), (1, 4, 24), (1, 4, 31)],
                    "f32": [(1, 4, 18), (1, 4, 22), (1, 4, 16), (1, 4, 25), (1, 16, 32)],
                    "bf16": [(1, 4, 31), (1, 4, 16), (1, 4, 27)]},
}


def _make(name):
    if name == "stencil27_128^3":
        return inputs.stencil3d(128, 128, 128, points=27, seed=1)
    if name == "fem3x3_n3M":
        return inputs.block_fem(1000000, bs=3, bmin=9, bmax=27, band_frac=0.05, seed=1)
    if name == "rmat_s22":
        return inputs.rmat(22, 16, 0.57, 0.19, 0.19, relabel=True, seed=1)
    return inputs.uniform(1000000, 1000000, 8, seed=1)


@pytest.fixture(scope="module", params=list(CASES))
def full(request, cuda_device):
    A = _make(request.param)
    x = inputs.vec_uniform(A.m, seed=0)
    yield request.param, A, x
    torch.cuda.empty_cache()


def _rounded(A, kind):
    vals = oracle.round_f32(A.values) if kind == "f32" else oracle.round_bf16(A.values)
    return inputs.CSR(A.n, A.m, A.rowptr, A.colidx, vals)


def _check_convert(M, B, rowptr, raw_values):
    got = M.export()
    assert got["nblocks"] == B.nblocks
    assert np.array_equal(got["block_rowptr"], B.block_rowptr)
    assert np.array_equal(got["block_colidx"], B.block_colidx)
    assert np.array_equal(got["block_masks"], B.block_masks)
    assert np.array_equal(got["values_raw"], raw_values)
    assert np.array_equal(got["valptr"], B.valptr(rowptr))
    return got


def test_float64_convert_and_spmv(full):
    name, A, x = full
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = spc5.upload_csr(A, torch.float64, "cuda")
    xd = torch.from_numpy(x).cuda()
    checked = set()
    for r, c, v in CASES[name]["f64"]:
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=v)
        if (r, c) not in checked:
            B = oracle.beta_convert(A, r, c)
            got = _check_convert(M, B, A.rowptr, B.values.view(np.uint64))
            if name == "rmat_s22" and r == 1:
                # hubs: intervals with more than 32 segments of 384 blocks take the fix-up's warp path
                assert got["nsegments"] > 0 and int(np.diff(B.block_rowptr).max()) > 32 * 384
            del B
            checked.add((r, c))
        buf = torch.full((A.n + 64,), float("nan"), dtype=torch.float64, device="cuda")
        M.spmv(xd, buf[:A.n])
        y = buf[:A.n].cpu().numpy()
        err = np.abs(y - y_ref)
        bad = err > TOL64 * absy
        assert not bad.any(), f"beta({r},{c}) variant {v}: {bad.sum()} rows over 1e-13 (|A||x|)_i"
        assert np.all(y[absy == 0] == 0)
        assert torch.isnan(buf[A.n:]).all(), "wrote past the end of y"
        M.destroy()
    del d


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_low_precision_convert_and_spmv(full, kind):
    name, A, x = full
    Ar = _rounded(A, kind)
    xr = oracle.round_f32(x)
    y_ref, absy = oracle.csr_spmv_dot2(Ar, xr)
    vdt = torch.float32 if kind == "f32" else torch.bfloat16
    vals = torch.from_numpy(Ar.values).to(vdt)
    rowptr = torch.from_numpy(np.ascontiguousarray(A.rowptr)).cuda()
    colidx = torch.from_numpy(np.ascontiguousarray(A.colidx)).cuda()
    vd = vals.cuda()
    xd = torch.from_numpy(xr).float().cuda()
    L = np.diff(A.rowptr).astype(np.float64)
    bound = (L + 1) * U32 / (1 - (L + 1) * U32) * absy
    checked = set()
    for r, c, v in CASES[name][kind]:
        M = spc5.convert(rowptr, colidx, vd, A.n, A.m, r, c, variant=v)
        if (r, c) not in checked:
            # the block structure depends only on the pattern; the values move as they are
            B = oracle.beta_convert(A, r, c)
            got = M.export()
            assert np.array_equal(got["block_colidx"], B.block_colidx)
            assert np.array_equal(got["block_masks"], B.block_masks)
            assert np.array_equal(got["block_rowptr"], B.block_rowptr)
            Br = oracle.beta_convert(Ar, r, c)
            want = torch.from_numpy(Br.values).to(vdt)
            want = want.view(torch.int32 if kind == "f32" else torch.int16).numpy()
            assert np.array_equal(got["values_raw"].view(want.dtype), want)
            del B, Br
            checked.add((r, c))
        y = M.spmv(xd).double().cpu().numpy()
        err = np.abs(y - y_ref)
        bad = err > bound + 1e-45
        assert not bad.any(), f"{kind} beta({r},{c}) variant {v}: {bad.sum()} rows over gamma_(L+1) (|A||x|)_i"
        M.destroy()


def test_spmm_full_size_stencil_k32(cuda_device):
    # the bench's SpMM workload: 27-point stencil 128^3, float32, k = 32, the
    # block-row tiles and the lane-per-row tiles; sampled columns against the oracle
    A = _make("stencil27_128^3")
    A = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, oracle.round_f32(A.values))
    k = 32
    X = oracle.round_f32(inputs.vec_uniform(A.m * k, seed=7).reshape(A.m, k))
    d = spc5.upload_csr(A, torch.float32, "cuda")
    Xd = torch.from_numpy(X).float().cuda()
    L = np.diff(A.rowptr).astype(np.float64)
    cols = (0, 13, 31)
    refs = {j: oracle.csr_spmv_dot2(A, np.ascontiguousarray(X[:, j])) for j in cols}
    for r, c, kt in ((2, 4, 32), (4, 8, 16), (8, 4, -32)):
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
        Y = M.spmm(Xd, ktile=kt).double().cpu().numpy()
        for j in cols:
            y_ref, absy = refs[j]
            assert np.all(np.abs(Y[:, j] - y_ref) <= (L + 1) * U32 / (1 - (L + 1) * U32) * absy + 1e-45), (r, c, kt, j)
        M.destroy()


def test_batch_full_size_256_matrices(cuda_device):
    # the bench's batched workload: 256 uneven float32 matrices in the shape and
    # variant the tuner picks; bit for bit against one product per matrix
    mats, keep, xs, ys, As = [], [], [], [], []
    for j in range(256):
        A = inputs.batch_matrix(j, seed=2)
        A = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, oracle.round_f32(A.values))
        As.append(A)
        d = spc5.upload_csr(A, torch.float32, "cuda")
        t = spc5.tune(d, reps=2)
        mats.append(spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, t["r"], t["c"], variant=t["variant"]))
        keep.append(d)
        xs.append(torch.rand(A.m, dtype=torch.float32, device="cuda"))
        ys.append(torch.full((A.n,), float("nan"), dtype=torch.float32, device="cuda"))
    B = spc5.Batch(mats, xs, ys)
    B.run()
    torch.cuda.synchronize()
    for j, M in enumerate(mats):
        single = M.spmv(xs[j])
        if M.variant in (22, 23, 32, 33) or 24 <= M.variant <= 29:
            # these variants sum in another order than the batch's one-lane
            # decode: both within the float32 bound of the oracle
            A = As[j]
            y_ref, absy = oracle.csr_spmv_dot2(A, xs[j].double().cpu().numpy())
            L = np.diff(A.rowptr).astype(np.float64)
            bound = (L + 1) * U32 / (1 - (L + 1) * U32) * absy + 1e-45
            assert np.all(np.abs(ys[j].double().cpu().numpy() - y_ref) <= bound), j
            assert np.all(np.abs(single.double().cpu().numpy() - y_ref) <= bound), j
        else:
            assert torch.equal(ys[j], single), j
    B.destroy()
    for M in mats:
        M.destroy()
