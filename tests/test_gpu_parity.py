"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Conversion must be bit-exact. float64 SpMV must satisfy
|y - y_ref|_i <= 1e-13 * (|A||x|)_i against the compensated (Dot2) oracle.
float32 / bfloat16 storage is checked against an oracle fed the same rounded
inputs, within the worst-case float32 summation bound gamma_{L_i+1} * (|A||x|)_i
(L_i = entries of row i; u = 2^-24), which holds for any summation order.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu

TOL64 = 1e-13


def _matrices():
    out = {
        "lap128": lambda: inputs.laplacian2d(128, 128),
        "rand_ragged": lambda: inputs.random_csr(301, 517, 0.03, seed=3),
        "st27_ragged": lambda: inputs.stencil3d(13, 11, 7, points=27, seed=4),
        "rmat11": lambda: inputs.rmat(11, seed=2),
        "uniform": lambda: inputs.uniform(3001, 2500, 8, seed=5),
        "fem": lambda: inputs.block_fem(700, seed=6),
        "dense64": lambda: inputs.CSR.from_dense(inputs.vec_normal(64 * 61, seed=8).reshape(64, 61)),
        "sparse_rows": lambda: inputs.random_csr(203, 90, 0.004, seed=9),  # mostly empty rows
    }
    return out


MATS = _matrices()
_cache = {}


def get(name):
    if name not in _cache:
        _cache[name] = MATS[name]()
    return _cache[name]


def dev_csr(A, dtype=torch.float64):
    return spc5.upload_csr(A, dtype, "cuda")


def guarded(n, dtype):
    """y with NaN guard cells after it; returns (buffer, view of length n)."""
    buf = torch.full((n + 64,), float("nan"), dtype=dtype, device="cuda")
    return buf, buf[:n]


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_convert_bit_exact(cuda_device, name, r, c):
    A = get(name)
    d = dev_csr(A)
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
    got = M.export()
    B = oracle.beta_convert(A, r, c)
    assert got["nblocks"] == B.nblocks
    assert np.array_equal(got["block_rowptr"], B.block_rowptr)
    assert np.array_equal(got["block_colidx"], B.block_colidx)
    assert np.array_equal(got["block_masks"], B.block_masks)
    assert np.array_equal(got["values_raw"], B.values.view(np.uint64))
    assert np.array_equal(got["valptr"], B.valptr(A.rowptr))
    M.destroy()


def check64(y, y_ref, absy):
    err = np.abs(y - y_ref)
    bad = err > TOL64 * absy
    assert not bad.any(), f"{bad.sum()} rows over tolerance; worst {err[bad].max()} vs {(TOL64 * absy)[bad].min()}"
    assert np.all(y[absy == 0] == 0)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_spmv_f64(cuda_device, name, r, c):
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
    xd = torch.from_numpy(x).cuda()
    buf, y = guarded(A.n, torch.float64)
    M.spmv(xd, y)
    torch.cuda.synchronize()
    check64(y.cpu().numpy(), y_ref, absy)
    assert torch.isnan(buf[A.n:]).all(), "wrote past the end of y"
    # the paper's accumulate form: y += A x
    y0 = inputs.vec_uniform(A.n, seed=1)
    yd = torch.from_numpy(y0.copy()).cuda()
    M.spmv_acc(xd, yd)
    ya = yd.cpu().numpy()
    err = np.abs(ya - (y0 + y_ref))
    assert np.all(err <= TOL64 * (absy + np.abs(y0)) + 1e-300)
    M.destroy()


VARIANTS = [1, 3, 5, 9, 10, 12, 13, 14, 15, 16, 17, 18, 19]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", ["st27_ragged", "rmat11", "fem", "sparse_rows"])
@pytest.mark.parametrize("r,c", [(1, 4), (1, 8), (2, 8), (4, 4), (4, 16), (8, 8), (8, 16)])
def test_spmv_variants(cuda_device, variant, name, r, c):
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=variant)
    check64(M.spmv(torch.from_numpy(x).cuda()).cpu().numpy(), y_ref, absy)
    M.destroy()


GROUP_VARIANTS = [22, 23]  # beta(1,c): two lanes per row, alternate stored values (natural, sorted order)


@pytest.mark.parametrize("variant", GROUP_VARIANTS)
@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("c", [4, 8, 16])
def test_spmv_group_variants(cuda_device, variant, name, c):
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    xd = torch.from_numpy(x).cuda()
    # default thresholds, and most rows on the segment path
    for lb, sb in [(0, 0), (1, 3)]:
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, c, variant=variant, long_blocks=lb, seg_blocks=sb)
        buf, y = guarded(A.n, torch.float64)
        M.spmv(xd, y)
        check64(y.cpu().numpy(), y_ref, absy)
        assert torch.isnan(buf[A.n:]).all(), "wrote past the end of y"
        assert torch.equal(M.spmv(xd), y)  # a fixed order
        y0 = inputs.vec_uniform(A.n, seed=1)
        yd = torch.from_numpy(y0.copy()).cuda()
        M.spmv_acc(xd, yd)
        assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)) + 1e-300)
        M.destroy()


@pytest.mark.parametrize("name", ["rmat11", "fem", "uniform", "sparse_rows"])
@pytest.mark.parametrize("window", [0, 32, 256, -1])
def test_sorted_two_lane_variant_matches_natural_bitwise(cuda_device, name, window):
    # variant 23 runs the two-lane row sum of variant 22 with rows taken in the
    # sorted work order: each row's arithmetic is unchanged, so the bits are
    A = get(name)
    d = dev_csr(A)
    xd = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
    for c in (4, 8):
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, c, variant=22, order_window=window, long_blocks=6)
        ref = M.spmv(xd).clone()
        M.set_variant(23)
        buf, y = guarded(A.n, torch.float64)
        M.spmv(xd, y)
        assert torch.equal(y, ref)
        assert torch.isnan(buf[A.n:]).all()
        M.destroy()


LANE_GROUP_VARIANTS = [24, 25, 26, 27, 28, 29]  # G = 4, 8, 16, 32 lanes per interval; 4, 8 in the sorted order


@pytest.mark.parametrize("variant", LANE_GROUP_VARIANTS)
@pytest.mark.parametrize("name", ["lap128", "rand_ragged", "st27_ragged", "rmat11", "fem", "dense64", "sparse_rows"])
@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_spmv_lane_group_variants(cuda_device, variant, name, r, c):
    # one lane per block, G lanes per interval: the float64 bound, the
    # accumulate form, no write past y, a fixed order; default thresholds and
    # most intervals on the segment path (long_blocks 2)
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    xd = torch.from_numpy(x).cuda()
    for lb in (0, 2):
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=variant, long_blocks=lb)
        buf, y = guarded(A.n, torch.float64)
        M.spmv(xd, y)
        check64(y.cpu().numpy(), y_ref, absy)
        assert torch.isnan(buf[A.n:]).all(), "wrote past the end of y"
        assert torch.equal(M.spmv(xd), y)
        y0 = inputs.vec_uniform(A.n, seed=1)
        yd = torch.from_numpy(y0.copy()).cuda()
        M.spmv_acc(xd, yd)
        assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)) + 1e-300)
        M.destroy()


@pytest.mark.parametrize("kind", ["f32", "bf16"])
@pytest.mark.parametrize("variant", LANE_GROUP_VARIANTS)
@pytest.mark.parametrize("name", ["st27_ragged", "rmat11", "fem", "uniform"])
def test_lane_group_variants_low_precision(cuda_device, kind, variant, name):
    A = get(name)
    Ar = rounded_case(A, kind)
    x = oracle.round_f32(inputs.vec_uniform(A.m, seed=0))
    y_ref, absy = oracle.csr_spmv_dot2(Ar, x)
    vdt = torch.float32 if kind == "f32" else torch.bfloat16
    vals = torch.from_numpy(Ar.values).to(vdt).cuda()
    rowptr, colidx = torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.colidx).cuda()
    L = np.diff(A.rowptr).astype(np.float64)
    u = 2.0**-24
    for r, c in [(1, 4), (1, 8), (2, 4), (4, 8), (8, 16)]:
        M = spc5.convert(rowptr, colidx, vals, A.n, A.m, r, c, variant=variant)
        y = M.spmv(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
        assert np.all(np.abs(y - y_ref) <= (L + 1) * u / (1 - (L + 1) * u) * absy + 1e-45), (r, c)
        M.destroy()


def test_lane_group_sorted_equals_natural_bitwise(cuda_device):
    # 28 / 29 run the row sums of 24 / 25 in another order of the intervals
    A = get("rmat11")
    d = dev_csr(A)
    xd = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
    for r, c in [(1, 4), (2, 8), (8, 4)]:
        for nat, srt in ((24, 28), (25, 29)):
            M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=nat, order_window=64)
            ref = M.spmv(xd).clone()
            M.set_variant(srt)
            assert torch.equal(M.spmv(xd), ref)
            M.destroy()


@pytest.mark.parametrize("name", ["lap128", "rand_ragged", "rmat11", "uniform", "fem", "sparse_rows", "dense64"])
@pytest.mark.parametrize("c", [4, 8, 16])
@pytest.mark.parametrize("lb", [0, 6])
def test_single_value_test_variants(cuda_device, name, c, lb):
    # Algorithm 2's test (variants 30 sorted, 31 natural): rows whose blocks
    # all hold one value are read like CSR, the others with the mask decode;
    # both add in storage order, so the bits equal the one-lane variants'
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    for vdt, xdt in ((torch.float64, torch.float64), (torch.float32, torch.float32), (torch.bfloat16, torch.float32)):
        d = dev_csr(A, vdt)
        xd = torch.from_numpy(x).to(xdt).cuda()
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, c, variant=5, long_blocks=lb)
        ref = M.spmv(xd).clone()
        for v in (30, 31):
            M.set_variant(v)
            buf, y = guarded(A.n, xdt)
            M.spmv(xd, y)
            assert torch.equal(y, ref), (v, vdt)
            assert torch.isnan(buf[A.n:]).all()
            if vdt == torch.float64:
                check64(y.cpu().numpy(), y_ref, absy)
                y0 = inputs.vec_uniform(A.n, seed=1)
                yd = torch.from_numpy(y0.copy()).cuda()
                M.spmv_acc(xd, yd)
                assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)) + 1e-300)
        M.destroy()


def _wide_rows():
    # rows of 80 to 600 entries in runs of 1 to 5 columns: blocks of one row
    # cover several 32-block trips of the streaming warp (carry between trips)
    rng = np.random.default_rng(11)
    n, m = 70, 4000
    rows, cols = [], []
    for i in range(n):
        if i % 9 == 4:
            continue  # an empty row now and then
        cs = set()
        target = int(rng.integers(80, 600))
        while len(cs) < target:
            start = int(rng.integers(0, m - 5))
            cs.update(range(start, start + int(rng.integers(1, 6))))
        cs = sorted(cs)[:target]
        rows += [i] * len(cs)
        cols += cs
    vals = inputs.vec_normal(len(cols), seed=12)
    dense = np.zeros((n, m))
    dense[np.array(rows), np.array(cols)] = vals
    return inputs.CSR.from_dense(dense)


@pytest.mark.parametrize("name", ["lap128", "rand_ragged", "st27_ragged", "rmat11", "uniform", "fem", "dense64",
                                  "sparse_rows", "wide_rows"])
@pytest.mark.parametrize("c", [4, 8, 16])
@pytest.mark.parametrize("lb", [0, 2, 100000])
def test_stream_variant(cuda_device, name, c, lb):
    # variant 32: the warp streams the blocks of its 32 rows, lane = block, a
    # segmented scan adds each row's run; warps holding a long row fall back
    # to one lane per row (long_blocks 2 sends most rows there), and with
    # long_blocks 100000 every row streams, carried across trips
    A = _wide_rows() if name == "wide_rows" else get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    xd = torch.from_numpy(x).cuda()
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, c, variant=32, long_blocks=lb)
    buf, y = guarded(A.n, torch.float64)
    M.spmv(xd, y)
    check64(y.cpu().numpy(), y_ref, absy)
    assert torch.isnan(buf[A.n:]).all(), "wrote past the end of y"
    assert torch.equal(M.spmv(xd), y)
    y0 = inputs.vec_uniform(A.n, seed=1)
    yd = torch.from_numpy(y0.copy()).cuda()
    M.spmv_acc(xd, yd)
    assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)) + 1e-300)
    M.destroy()
    L = np.diff(A.rowptr).astype(np.float64)
    u = 2.0**-24
    for kind in ("f32", "bf16"):
        Ar = rounded_case(A, kind)
        xr = oracle.round_f32(x)
        yr_ref, absr = oracle.csr_spmv_dot2(Ar, xr)
        vals = torch.from_numpy(Ar.values).to(torch.float32 if kind == "f32" else torch.bfloat16).cuda()
        M = spc5.convert(d.rowptr, d.colidx, vals, A.n, A.m, 1, c, variant=32, long_blocks=lb)
        buf, y = guarded(A.n, torch.float32)
        M.spmv(torch.from_numpy(xr).float().cuda(), y)
        assert np.all(np.abs(y.double().cpu().numpy() - yr_ref) <= (L + 1) * u / (1 - (L + 1) * u) * absr + 1e-45)
        assert torch.isnan(buf[A.n:]).all()
        M.destroy()


def test_stream_variant_needs_r1(cuda_device):
    A = get("fem")
    d = dev_csr(A)
    with pytest.raises(spc5.Spc5Error) as ei:
        spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 4, variant=32)
    assert ei.value.status == spc5.EUNSUPPORTED


@pytest.mark.parametrize("name", ["lap128", "rand_ragged", "rmat11", "uniform", "fem", "sparse_rows", "dense64"])
@pytest.mark.parametrize("c", [4, 8, 16])
@pytest.mark.parametrize("lb", [0, 6])
def test_two_lane_single_value_variant(cuda_device, name, c, lb):
    # variant 33: two lanes per row, rows whose blocks all hold one value read
    # like a two-lane CSR kernel (Algorithm 2's test); lane g still takes the
    # values of rank g, g + 2, ..., so the bits equal variant 22's
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    for vdt, xdt in ((torch.float64, torch.float64), (torch.float32, torch.float32), (torch.bfloat16, torch.float32)):
        d = dev_csr(A, vdt)
        xd = torch.from_numpy(x).to(xdt).cuda()
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, c, variant=22, long_blocks=lb)
        ref = M.spmv(xd).clone()
        M.set_variant(33)
        buf, y = guarded(A.n, xdt)
        M.spmv(xd, y)
        assert torch.equal(y, ref), vdt
        assert torch.isnan(buf[A.n:]).all()
        if vdt == torch.float64:
            check64(y.cpu().numpy(), y_ref, absy)
            y0 = inputs.vec_uniform(A.n, seed=1)
            yd = torch.from_numpy(y0.copy()).cuda()
            M.spmv_acc(xd, yd)
            assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)) + 1e-300)
        M.destroy()


def test_single_value_class_needs_r1(cuda_device):
    A = get("rmat11")
    d = dev_csr(A)
    for v in (30, 31, 33):
        with pytest.raises(spc5.Spc5Error) as ei:
            spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 8, variant=v)
        assert ei.value.status == spc5.EUNSUPPORTED


def test_group_variants_low_precision_and_limits(cuda_device):
    # dyadic Laplacian: exact partial sums, so any order gives the oracle's bits
    A = get("lap128")
    x = inputs.vec_dyadic(A.m, seed=0, bits=20)
    y_ref = oracle.csr_spmv(A, x)
    for vdt, xdt in [(torch.float64, torch.float64), (torch.float32, torch.float32), (torch.bfloat16, torch.float32)]:
        d = dev_csr(A, vdt)
        for v in GROUP_VARIANTS:
            M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8, variant=v)
            y = M.spmv(torch.from_numpy(x).to(xdt).cuda()).double().cpu().numpy()
            assert np.array_equal(y, y_ref), (vdt, v)
            M.destroy()
    # float32 storage on a ragged matrix: the worst-case float32 summation bound
    B = get("rmat11")
    rv = oracle.round_f32(B.values)
    xr = oracle.round_f32(inputs.vec_uniform(B.m, seed=0))
    y_ref, absy = oracle.csr_spmv_dot2(inputs.CSR(B.n, B.m, B.rowptr, B.colidx, rv), xr)
    vals = torch.from_numpy(rv).float().cuda()
    L = np.diff(B.rowptr).astype(np.float64)
    u = 2.0**-24
    for v in GROUP_VARIANTS:
        M = spc5.convert(torch.from_numpy(B.rowptr).cuda(), torch.from_numpy(B.colidx).cuda(), vals, B.n, B.m, 1, 4,
                         variant=v)
        y = M.spmv(torch.from_numpy(xr).float().cuda()).double().cpu().numpy()
        assert np.all(np.abs(y - y_ref) <= (L + 1) * u / (1 - (L + 1) * u) * absy + 1e-45)
        M.destroy()
    # r > 1: refused at conversion and when switching
    d = dev_csr(B)
    with pytest.raises(spc5.Spc5Error) as ei:
        spc5.convert(d.rowptr, d.colidx, d.values, B.n, B.m, 2, 4, variant=22)
    assert ei.value.status == spc5.EUNSUPPORTED
    M = spc5.convert(d.rowptr, d.colidx, d.values, B.n, B.m, 4, 8)
    for v in GROUP_VARIANTS:
        with pytest.raises(spc5.Spc5Error) as ei:
            M.set_variant(v)
        assert ei.value.status == spc5.EUNSUPPORTED
    M.destroy()


@pytest.mark.parametrize("name", ["st27_ragged", "rmat11", "fem", "uniform"])
@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_variants_sum_in_the_same_order(cuda_device, name, r, c):
    # every short-interval variant adds a row's products in storage order, so
    # all of them give the same bits; the segment path (its own fixed order)
    # is the same in all variants
    A = get(name)
    d = dev_csr(A)
    xd = torch.from_numpy(inputs.vec_normal(A.m, seed=3)).cuda()
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=8)
    ref = M.spmv(xd).clone()
    for v in VARIANTS:
        M.set_variant(v)
        assert torch.equal(M.spmv(xd), ref), v
    M.destroy()
    # one sorting window over all intervals, and larger segments
    for v, sb in [(10, 0), (13, 0), (15, 64), (13, 3)]:
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=8, seg_blocks=sb, variant=v,
                         order_window=-1)
        y = M.spmv(xd)
        if sb == 0:
            assert torch.equal(y, ref), v
        else:  # other segment boundaries: same values up to the summation order
            y_ref, absy = oracle.csr_spmv_dot2(A, xd.cpu().numpy())
            check64(y.cpu().numpy(), y_ref, absy)
        M.destroy()


@pytest.mark.parametrize("r,c", [(1, 4), (2, 8), (8, 16)])
def test_sorted_order_device_and_host_sorts(cuda_device, r, c):
    # windows of up to 4096 intervals are sorted on the device, larger ones
    # (or all intervals together) on the host; every order must cover each
    # short interval once, so y is bit for bit that of the natural order
    A = inputs.rmat(14, seed=7)  # 16,384 rows, power-law lengths
    x = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
    d = dev_csr(A)
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=5)
    ref = M.spmv(x).clone()
    M.destroy()
    I = (A.n + r - 1) // r
    for ow in (1, 33, 1024, 4096 * r, 4096 * r + r, -1):
        for v in (10, 13):
            M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=v, order_window=ow)
            assert torch.equal(M.spmv(x), ref), (ow, v, I)
            M.destroy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autotune_keeps_a_candidate_and_the_result(cuda_device, dtype):
    A = get("rmat11")
    vals = A.values if dtype == torch.float64 else oracle.round_f32(A.values)
    d = dev_csr(inputs.CSR(A.n, A.m, A.rowptr, A.colidx, vals), dtype)
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8)
    xd = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).to(torch.float64 if dtype == torch.float64 else torch.float32).cuda()
    ref = M.spmv(xd).clone()
    y = torch.empty_like(ref)
    v, ms = M.autotune(xd, y, reps=3)
    cands = ((5, 10, 13, 15) if dtype == torch.float64 else (5, 10, 13, 15, 16, 18, 32)) + (22, 23, 30, 33)
    assert v in cands and ms > 0
    got = M.spmv(xd)
    if v < 20 or v == 30:
        assert torch.equal(got, ref)  # variants 0-19 and 30 add in the same order
    else:  # two lanes per row, the streaming warp: their own fixed orders
        Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, vals)
        y_ref, absy = oracle.csr_spmv_dot2(Ar, xd.double().cpu().numpy())
        L = np.diff(A.rowptr).astype(np.float64)
        tol = TOL64 if dtype == torch.float64 else (L + 1) * 2.0**-23
        assert np.all(np.abs(got.double().cpu().numpy() - y_ref) <= tol * absy + 1e-45)
    M.destroy()


@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_long_interval_segments(cuda_device, r, c):
    # force every interval with more than one block onto the segment path
    A = get("rmat11")
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    xd = torch.from_numpy(x).cuda()
    for lb, sb in [(1, 1), (1, 3), (2, 7), (4, 64)]:
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, long_blocks=lb, seg_blocks=sb)
        assert M.export()["nsegments"] > 0
        check64(M.spmv(xd).cpu().numpy(), y_ref, absy)
        y0 = inputs.vec_uniform(A.n, seed=1)
        yd = torch.from_numpy(y0.copy()).cuda()
        M.spmv_acc(xd, yd)
        assert np.all(np.abs(yd.cpu().numpy() - (y0 + y_ref)) <= TOL64 * (absy + np.abs(y0)))
        M.destroy()


@pytest.mark.parametrize("r,c", spc5.SHAPES)
def test_dyadic_config_bit_exact_all_precisions(cuda_device, r, c):
    # 5-point Laplacian with x = k / 2^20: every partial sum is exact in float32
    # and float64, and the values 4 / -1 are exact in bfloat16, so every format
    # and precision reproduces the oracle bit for bit.
    A = get("lap128")
    x = inputs.vec_dyadic(A.m, seed=0, bits=20)
    y_ref = oracle.csr_spmv(A, x)
    for vdt, xdt in [(torch.float64, torch.float64), (torch.float32, torch.float32), (torch.bfloat16, torch.float32)]:
        d = dev_csr(A, vdt)
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
        y = M.spmv(torch.from_numpy(x).to(xdt).cuda()).double().cpu().numpy()
        assert np.array_equal(y, y_ref), (vdt, np.abs(y - y_ref).max())
        M.destroy()


def rounded_case(A, kind):
    """Values rounded to the storage type and x to float32, on the host."""
    rv = oracle.round_f32(A.values) if kind == "f32" else oracle.round_bf16(A.values)
    Ar = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, rv)
    return Ar


@pytest.mark.parametrize("kind", ["f32", "bf16"])
@pytest.mark.parametrize("name", ["st27_ragged", "rmat11", "uniform", "fem", "rand_ragged"])
@pytest.mark.parametrize("r,c", [(1, 8), (2, 4), (4, 8), (8, 16), (1, 16), (8, 4)])
def test_spmv_low_precision(cuda_device, kind, name, r, c):
    A = get(name)
    Ar = rounded_case(A, kind)
    x = oracle.round_f32(inputs.vec_uniform(A.m, seed=0))
    y_ref, absy = oracle.csr_spmv_dot2(Ar, x)
    vdt = torch.float32 if kind == "f32" else torch.bfloat16
    vals = torch.from_numpy(Ar.values).to(vdt)  # exact: values are representable
    assert np.array_equal(vals.double().numpy(), Ar.values)
    rowptr = torch.from_numpy(A.rowptr).cuda()
    colidx = torch.from_numpy(A.colidx).cuda()
    M = spc5.convert(rowptr, colidx, vals.cuda(), A.n, A.m, r, c)
    y = M.spmv(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    L = np.diff(A.rowptr).astype(np.float64)
    u = 2.0**-24
    bound = (L + 1) * u / (1 - (L + 1) * u) * absy
    assert np.all(np.abs(y - y_ref) <= bound + 1e-45)
    # error against the float64 oracle on unrounded values (reported, loosely bounded)
    y64, abs64 = oracle.csr_spmv_dot2(A, inputs.vec_uniform(A.m, seed=0))
    rel = np.abs(y - y64) / np.maximum(abs64, 1e-300)
    store = 2.0**-8 if kind == "bf16" else u  # unit roundoff of the storage type (8 / 24 significand bits)
    assert np.all(rel <= store + (L + 3) * u + 1e-12)
    M.destroy()


@pytest.mark.parametrize("group", [0, 1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("name", ["lap128", "st27_ragged", "rmat11", "sparse_rows", "fem"])
def test_csr_kernel(cuda_device, name, group):
    A = get(name)
    x = inputs.vec_uniform(A.m, seed=0)
    y_ref, absy = oracle.csr_spmv_dot2(A, x)
    d = dev_csr(A)
    y = spc5.csr_spmv(d.rowptr, d.colidx, d.values, A.n, A.m, torch.from_numpy(x).cuda(), group=group)
    check64(y.cpu().numpy(), y_ref, absy)
    Ar = rounded_case(A, "f32")
    xr = oracle.round_f32(x)
    y_ref32, absy32 = oracle.csr_spmv_dot2(Ar, xr)
    y = spc5.csr_spmv(d.rowptr, d.colidx, torch.from_numpy(Ar.values).float().cuda(), A.n, A.m,
                      torch.from_numpy(xr).float().cuda(), group=group).double().cpu().numpy()
    L = np.diff(A.rowptr).astype(np.float64)
    u = 2.0**-24
    assert np.all(np.abs(y - y_ref32) <= (L + 1) * u / (1 - (L + 1) * u) * absy32 + 1e-45)


@pytest.mark.parametrize("r", [1, 2])
def test_invalid_csr_is_rejected_with_codes(cuda_device, r):
    def attempt(rowptr, colidx, m):
        rp = torch.tensor(rowptr, dtype=torch.int64, device="cuda")
        ci = torch.tensor(colidx, dtype=torch.int32, device="cuda")
        v = torch.ones(len(colidx), dtype=torch.float64, device="cuda")
        try:
            spc5.convert(rp, ci, v, len(rowptr) - 1, m, r, 4)
        except spc5.Spc5Error as e:
            return e.status
        return spc5.OK

    assert attempt([0, 3, 2], [0, 1, 2], 4) == spc5.EINVAL  # row pointer going backwards
    assert attempt([0, 2, 2], [0, 1, 2], 4) == spc5.EINVAL  # last pointer is not nnz
    # errors past the first entries of long rows are found too
    assert attempt([0, 40, 41], list(range(20)) + list(range(21, 41)) + [7], 64) == spc5.OK
    assert attempt([0, 40, 41], list(range(20)) + [30] + list(range(21, 40)) + [7], 64) == spc5.EUNSORTED

    assert attempt([0, 2, 3], [1, 2, 0], 4) == spc5.OK
    assert attempt([0, 2, 3], [2, 1, 0], 4) == spc5.EUNSORTED
    assert attempt([0, 2, 3], [1, 1, 0], 4) == spc5.EDUP
    assert attempt([0, 2, 3], [1, 2, 4], 4) == spc5.ERANGE
    assert attempt([0, 2, 3], [1, 2, -1], 4) == spc5.ERANGE
    # the first bad row decides the code
    assert attempt([0, 2, 4], [1, 1, 3, 2], 4) == spc5.EDUP


def test_empty_and_degenerate(cuda_device):
    # no entries at all
    A = inputs.CSR(37, 20, np.zeros(38, np.int64), np.zeros(0, np.int32), np.zeros(0))
    d = dev_csr(A)
    for r, c in [(1, 4), (8, 16)]:
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
        y = M.spmv(torch.ones(20, dtype=torch.float64, device="cuda"))
        assert torch.count_nonzero(y).item() == 0
        M.destroy()
    # one row, one column
    B = inputs.CSR(1, 1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([3.0]))
    d = dev_csr(B)
    M = spc5.convert(d.rowptr, d.colidx, d.values, 1, 1, 8, 16)
    assert M.spmv(torch.tensor([2.0], dtype=torch.float64, device="cuda")).item() == 6.0
    # identity and permutation reproduce x exactly
    n = 1000
    x = inputs.vec_normal(n, seed=3)
    perm = np.random.default_rng(1).permutation(n)
    P = inputs.CSR(n, n, np.arange(n + 1, dtype=np.int64), perm.astype(np.int32), np.ones(n))
    Pd = dev_csr(P)
    for r, c in spc5.SHAPES:
        M = spc5.convert(Pd.rowptr, Pd.colidx, Pd.values, n, n, r, c)
        assert np.array_equal(M.spmv(torch.from_numpy(x).cuda()).cpu().numpy(), x[perm])
        M.destroy()


def test_count_blocks_matches_oracle(cuda_device):
    for name in ["lap128", "rmat11", "st27_ragged", "rand_ragged"]:
        A = get(name)
        d = dev_csr(A)
        got = spc5.count_blocks(d.rowptr, d.colidx, A.n, A.m)
        want = [oracle.beta_count(A, r, c)[1] for r, c in spc5.SHAPES]
        assert list(got) == want


def _long_rows_csr():
    # rows far longer than the chunked counting threshold: sparse random,
    # one dense run, and clusters with gaps around c
    rng = np.random.default_rng(5)
    m = 200_000
    rows = []
    for i in range(64):
        if i == 5:
            cols = rng.choice(m, 30_000, replace=False)
        elif i == 6:
            cols = np.arange(1000, 21_000)
        elif i == 7:
            starts = np.cumsum(rng.integers(5, 21, 6000)) + 3
            cols = np.unique(np.concatenate([starts, starts + 1, starts + 2]))
            cols = cols[cols < m]
        elif i in (4, 13):  # neighbours of the long rows inside their intervals
            cols = rng.choice(m, 9000, replace=False)
        else:
            cols = rng.choice(m, rng.integers(0, 40), replace=False)
        rows.append(np.sort(cols).astype(np.int32))
    rowptr = np.zeros(65, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.concatenate(rows)
    return inputs.CSR(64, m, rowptr, colidx, np.ones(colidx.size))


def test_count_blocks_long_rows_match_oracle(cuda_device):
    A = _long_rows_csr()
    d = dev_csr(A)
    got = spc5.count_blocks(d.rowptr, d.colidx, A.n, A.m)
    want = [oracle.beta_count(A, r, c)[1] for r, c in spc5.SHAPES]
    assert list(got) == want
    f = spc5.features(d)
    assert np.allclose(f[:12], [A.nnz / w for w in want], rtol=0, atol=0)


def test_copy_kernel(cuda_device):
    a = torch.randint(0, 2**31, (1 << 20,), dtype=torch.int32, device="cuda")
    b = torch.zeros_like(a)
    spc5.copy(a, b)
    assert torch.equal(a, b)


def test_pool_trim_between_conversions(cuda_device):
    # handle memory kept by the library's pool is reused, and can be handed back
    A = get("fem")
    d = dev_csr(A)
    x = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).cuda()
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8)
    ref = M.spmv(x).clone()
    M.destroy()
    for _ in range(2):
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 1, 8)
        assert torch.equal(M.spmv(x), ref)
        M.destroy()
        spc5.pool_trim()
