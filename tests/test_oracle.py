"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own code: brute force on tiny
inputs, exact rational arithmetic, closed forms, values printed in the paper
(tests/golden/, each with its citation) and hand-derived counts.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1801_01134_gb300 import inputs
from tests.conftest import read_golden


def popcount_bytes(a: np.ndarray) -> int:
    return int(np.unpackbits(np.asarray(a, dtype=np.uint8)).sum())


def csr_of_dense(D):
    return inputs.CSR.from_dense(D)


def tiny_random(n, m, density, seed):
    A = inputs.random_csr(n, m, density, seed)
    assert oracle.validate(A)[0] == oracle.OK
    return A


# ---------------------------------------------------------------- generators

def test_generator_is_counter_based_and_seeded():
    a = inputs.raw_u64(1000, seed=7, stream=3)
    b = inputs.raw_u64(1000, seed=7, stream=3)
    c = inputs.raw_u64(1000, seed=8, stream=3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    u = inputs.vec_uniform(200000, seed=0)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01
    z = inputs.vec_normal(200000, seed=0)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_splitmix_mix_is_a_bijection_sample():
    # the SplitMix64 finaliser is invertible: distinct inputs give distinct outputs
    outs = {inputs.splitmix_mix(i) for i in range(5000)}
    assert len(outs) == 5000


def test_dyadic_vector_is_exact_in_float32():
    x = inputs.vec_dyadic(10000, seed=0, bits=20)
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)
    assert np.all(np.abs(x) <= 1.0)
    assert np.array_equal(x * 2**20, np.round(x * 2**20))


def test_laplacian2d_shape_and_row_sums():
    A = inputs.laplacian2d(128, 128)
    assert A.n == 16384 and A.nnz == 81408  # 5n - 2*128 - 2*128
    y = oracle.csr_spmv(A, np.ones(A.n))
    grid = y.reshape(128, 128)
    assert np.all(grid[1:-1, 1:-1] == 0.0)  # interior rows of the Laplacian sum to zero
    assert grid[0, 0] == 2.0 and grid[0, 5] == 1.0


@pytest.mark.parametrize("dims", [(5, 4, 3), (8, 8, 8)])
def test_stencil_nnz_closed_forms(dims):
    nx, ny, nz = dims
    A27 = inputs.stencil3d(nx, ny, nz, points=27)
    assert A27.nnz == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)
    A7 = inputs.stencil3d(nx, ny, nz, points=7, normal_values=False)
    n = nx * ny * nz
    assert A7.nnz == 7 * n - 2 * (nx * ny + ny * nz + nx * nz)
    for A in (A27, A7):
        assert oracle.validate(A)[0] == oracle.OK


def test_block_fem_structure():
    A = inputs.block_fem(2000, bs=3, bmin=9, bmax=27, band_frac=0.05, seed=1)
    assert oracle.validate(A)[0] == oracle.OK
    lens = np.diff(A.rowptr)
    assert np.all(lens % 3 == 0) and lens.min() >= 27 and lens.max() <= 81
    # rows of one block row share their pattern; columns come in aligned triples
    assert np.all(A.colidx[::3] % 3 == 0)


def test_rmat_and_uniform_structure():
    R = inputs.rmat(12, edge_factor=16, seed=1)
    assert R.n == 4096 and oracle.validate(R)[0] == oracle.OK
    assert 0.5 * 16 * 4096 < R.nnz <= 16 * 4096  # duplicates dropped
    lens = np.diff(R.rowptr)
    assert lens.max() > 10 * lens.mean()  # power-law degrees
    U = inputs.uniform(5000, 5000, 8, seed=1)
    assert U.nnz == 40000 and np.all(np.diff(U.rowptr) == 8)
    assert oracle.validate(U)[0] == oracle.OK


# ------------------------------------------------------------------ CSR SpMV

@pytest.mark.parametrize("seed", range(6))
def test_csr_spmv_matches_dense_gemv_bruteforce(seed):
    n, m = [(1, 1), (7, 5), (13, 17), (32, 9), (40, 64), (64, 64)][seed]
    A = tiny_random(n, m, 0.3, seed)
    x = inputs.vec_uniform(m, seed=seed)
    D = A.to_dense()
    y_ref = oracle.dense_gemv(D, x)
    y = oracle.csr_spmv(A, x)
    yd, _ = oracle.csr_spmv_dot2(A, x)
    scale = np.abs(D) @ np.abs(x)
    assert np.all(np.abs(y - y_ref) <= 1e-14 * scale + 0.0)
    assert np.all(np.abs(yd - y_ref) <= 1e-14 * scale + 0.0)


def test_identity_and_permutation_are_exact():
    n = 257
    x = inputs.vec_normal(n, seed=3)
    I = csr_of_dense(np.eye(n))
    assert np.array_equal(oracle.csr_spmv(I, x), x)
    perm = np.random.default_rng(0).permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    assert np.array_equal(oracle.csr_spmv(csr_of_dense(P), x), x[perm])
    assert np.array_equal(oracle.csr_spmv_dot2(csr_of_dense(P), x)[0], x[perm])


def exact_dot(vals, xs):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(vals, xs)), Fraction(0))


def test_dot2_against_exact_rational_arithmetic():
    rng = np.random.default_rng(5)
    for trial in range(40):
        k = int(rng.integers(1, 60))
        # ill-conditioned rows: large cancelling terms plus small ones
        vals = rng.standard_normal(k) * (10.0 ** rng.integers(-8, 9, size=k))
        xs = rng.standard_normal(k)
        if k > 2:
            vals[1] = -vals[0] * xs[0] / xs[1]
        D = vals.reshape(1, k)
        A = csr_of_dense(D)
        keep = A.colidx
        yd, absy = oracle.csr_spmv_dot2(A, xs)
        ex = exact_dot(vals[keep], xs[keep])
        err = abs(Fraction(float(yd[0])) - ex)
        # Dot2 bound (Ogita, Rump & Oishi 2005, Prop. 5.5): u|exact| + gamma_{n}^2 sum|a||x|
        u = 2.0**-53
        g = k * u / (1 - k * u)
        bound = Fraction(u) * abs(ex) + Fraction(g * g) * Fraction(float(absy[0]))
        assert err <= bound * 2, (trial, float(err), float(bound))


def test_dot2_beats_naive_on_cancellation():
    A = csr_of_dense(np.array([[1e16, 1.0, -1e16]]))
    x = np.ones(3)
    assert oracle.csr_spmv_dot2(A, x)[0][0] == 1.0
    assert oracle.csr_spmv(A, x)[0] != 1.0  # the plain loop loses the 1


def test_validate_rejects_bad_csr():
    good = tiny_random(10, 10, 0.4, 1)
    assert oracle.validate(good)[0] == oracle.OK

    class M:
        pass

    def mk(rowptr, colidx, m=10):
        a = M()
        a.n, a.m = len(rowptr) - 1, m
        a.rowptr, a.colidx = np.array(rowptr, np.int64), np.array(colidx, np.int32)
        a.values = np.zeros(len(colidx))
        return a

    assert oracle.validate(mk([0, 3], [1, 5, 3])) == (oracle.EUNSORTED, 0)
    assert oracle.validate(mk([0, 1, 3], [1, 4, 4])) == (oracle.EDUP, 1)
    assert oracle.validate(mk([0, 2], [1, 10])) == (oracle.ERANGE, 0)
    assert oracle.validate(mk([0, 2], [-1, 3])) == (oracle.ERANGE, 0)


# --------------------------------------------------------------- beta(r,c)

def test_vexpand_worked_example():
    rows = read_golden("vexpand_example.txt")
    mask = int(rows[0][1], 2)
    lanes = [int(v) for v in rows[1][1:]]
    cols = [k for k in range(8) if (mask >> k) & 1]
    p = np.array([10.0, 20.0, 30.0, 40.0])
    D = np.zeros((1, 8))
    D[0, cols] = p
    B = oracle.beta_convert(csr_of_dense(D), 1, 8)
    assert B.nblocks == 1 and B.block_colidx[0] == 0
    assert int(B.block_masks[0]) == mask
    assert np.array_equal(B.values, p)
    # the product with x = unit vector e_k reads lane k of the expanded vector
    for k in range(8):
        x = np.zeros(8)
        x[k] = 1.0
        want = 0.0 if lanes[k] < 0 else p[lanes[k]]
        assert oracle.beta_spmv(B, x)[0] == want


def check_beta_invariants(A, B):
    r, c = B.r, B.c
    mb = oracle.mask_bytes(r, c)
    I = oracle.n_intervals(A.n, r)
    assert B.block_rowptr.shape == (I + 1,) and B.block_rowptr[0] == 0
    assert np.all(np.diff(B.block_rowptr) >= 0)
    assert B.block_masks.shape == (B.nblocks * mb,)
    assert popcount_bytes(B.block_masks) == A.nnz
    bits = np.unpackbits(B.block_masks.reshape(-1, mb) if B.nblocks else np.zeros((0, mb), np.uint8),
                         axis=1, bitorder="little")[:, : r * c]
    if B.nblocks:
        assert np.all(bits.sum(axis=1) >= 1)  # no empty block
        colmask = bits.reshape(-1, r, c).any(axis=1)
        assert np.all(colmask[:, 0])  # a block starts at a column holding a nonzero
    for it in range(I):
        s, e = B.block_rowptr[it], B.block_rowptr[it + 1]
        starts = B.block_colidx[s:e]
        assert np.all(np.diff(starts) >= c)  # blocks of an interval are disjoint, left to right
        rows_here = min(r, A.n - it * r)
        if B.nblocks and rows_here < r:
            assert not bits[s:e].reshape(-1, r, c)[:, rows_here:, :].any()
        if e > s:
            over = starts[:, None] + np.arange(c)[None, :] >= A.m
            assert not bits[s:e].reshape(-1, r, c)[np.broadcast_to(over[:, None, :], (e - s, r, c))].any()


@pytest.mark.parametrize("r,c", oracle.SHAPES)
def test_roundtrip_bit_exact_all_shapes(r, c):
    for seed, (n, m, d) in enumerate([(37, 41, 0.15), (64, 64, 0.05), (50, 200, 0.3), (9, 3, 0.6)]):
        A = tiny_random(n, m, d, 100 + seed)
        B = oracle.beta_convert(A, r, c)
        check_beta_invariants(A, B)
        C = oracle.beta_expand(B)
        assert np.array_equal(C.rowptr, A.rowptr)
        assert np.array_equal(C.colidx, A.colidx)
        assert np.array_equal(C.values.view(np.uint64), A.values.view(np.uint64))


@pytest.mark.parametrize("r,c", oracle.SHAPES)
def test_beta_spmv_equals_plain_csr_bitwise(r, c):
    # the blocks of an interval are disjoint and stored left to right, so the
    # product read from the beta arrays adds each row's entries in ascending
    # column order, as the plain CSR loop does: identical float64 results.
    A = inputs.stencil3d(9, 7, 5, points=27, seed=4)
    x = inputs.vec_uniform(A.m, seed=0)
    B = oracle.beta_convert(A, r, c)
    check_beta_invariants(A, B)
    assert np.array_equal(oracle.beta_spmv(B, x), oracle.csr_spmv(A, x))
    # the paper's kernels accumulate into y
    y0 = inputs.vec_uniform(A.n, seed=9)
    assert np.allclose(oracle.beta_spmv(B, x, y0), y0 + oracle.csr_spmv(A, x), rtol=0, atol=1e-13)


@pytest.mark.parametrize("r,c", [(1, 4), (2, 8), (4, 4), (8, 16)])
def test_beta_spmv_matches_dense_gemv_bruteforce(r, c):
    # n not a multiple of r (a ragged last interval) and columns near m - 1 (blocks
    # running past the last column): the product read from the beta arrays must
    # equal the textbook dense sum on every row
    rng = np.random.default_rng(40 + r * c)
    for n, m in ((13, 11), (9, 30), (3, 5)):
        D = np.where(rng.random((n, m)) < 0.35, rng.standard_normal((n, m)), 0.0)
        x = rng.standard_normal(m)
        B = oracle.beta_convert(csr_of_dense(D), r, c)
        got = oracle.beta_spmv(B, x)
        assert np.allclose(got, oracle.dense_gemv(D, x), rtol=1e-14, atol=1e-14)
        # a nonzero moved to another place changes the product there
        if B.nnz:
            B2 = oracle.Beta(B.n, B.m, B.r, B.c, B.block_rowptr, B.block_colidx, B.block_masks, B.values * 2.0)
            assert np.allclose(oracle.beta_spmv(B2, x), 2.0 * got, rtol=1e-14, atol=1e-14)


def min_cover_bruteforce(colsets, c):
    """Minimum number of c-wide windows covering the union of the given column sets."""
    cols = sorted(set().union(*colsets))
    if not cols:
        return 0
    best = len(cols)
    # windows only need to start at a column holding a nonzero
    for k in range(1, len(cols) + 1):
        for starts in itertools.combinations(cols, k):
            if all(any(s <= q < s + c for s in starts) for q in cols):
                return k
    return best


def test_greedy_block_count_is_minimum_cover():
    rng = np.random.default_rng(11)
    for trial in range(150):
        r = int(rng.choice([1, 2, 4]))
        c = int(rng.choice([4, 8]))
        m = int(rng.integers(1, 13))
        D = (rng.random((r, m)) < rng.uniform(0.1, 0.7)).astype(float)
        A = csr_of_dense(D)
        counts, nb = oracle.beta_count(A, r, c)
        colsets = [set(np.nonzero(D[i])[0].tolist()) for i in range(r)]
        assert nb == min_cover_bruteforce(colsets, c), (trial, D.tolist(), r, c)


def test_identity_blocks():
    n = 64
    A = csr_of_dense(np.eye(n))
    for r, c in oracle.SHAPES:
        B = oracle.beta_convert(A, r, c)
        per = math.ceil(r / c)
        assert B.nblocks == oracle.n_intervals(n, r) * per
        if r <= c:
            assert np.array_equal(B.block_colidx, np.arange(0, n, r))
            mb = oracle.mask_bytes(r, c)
            want = sum(1 << (i * c + i) for i in range(r))
            got = int.from_bytes(bytes(B.block_masks[:mb]), "little")
            assert got == want


def test_r1_keeps_csr_values():
    A = inputs.uniform(300, 500, 9, seed=2)
    for c in (4, 8, 16):
        B = oracle.beta_convert(A, 1, c)
        assert np.array_equal(B.values, A.values)


def test_laplacian128_block_counts_hand_derived():
    A = inputs.laplacian2d(128, 128)
    for r, c, nb in read_golden("laplacian128_blocks.txt"):
        assert oracle.beta_count(A, int(r), int(c))[1] == int(nb)


def test_table1_avg_rows():
    rows = {row[0]: [float(v) for v in row[1:]] for row in read_golden("table1_avg.txt")}
    A = inputs.stencil3d(32, 32, 32, points=7, normal_values=False)
    got = [A.nnz / oracle.beta_count(A, r, c)[1] for r, c in oracle.PAPER_SHAPES]
    assert np.all(np.abs(np.array(got) - np.array(rows["atmosmodd"])) <= 0.1 + 1e-9), got
    Dn = csr_of_dense(np.ones((64, 64)))
    got = [Dn.nnz / oracle.beta_count(Dn, r, c)[1] for r, c in oracle.PAPER_SHAPES]
    assert got == rows["Dense-8000"]


def test_occupancy_eq1_matches_array_sizes_and_eq4_break_even():
    for A in (inputs.stencil3d(12, 12, 12, points=27), inputs.uniform(2000, 2000, 5, seed=3),
              inputs.rmat(10, seed=2)):
        for r, c in oracle.SHAPES:
            B = oracle.beta_convert(A, r, c)
            if (r * c) % 8 == 0:
                arrays = (B.values.nbytes + B.block_colidx.nbytes + B.block_masks.nbytes
                          + B.block_rowptr.nbytes)
                assert arrays == oracle.occupancy_beta(A.n, A.nnz, B.nblocks, r, c)
            # Eq. 4 compares the per-block index bytes with the per-entry CSR colidx
            beta_idx = B.nblocks * (4 + r * c / 8)
            csr_idx = A.nnz * 4
            assert (beta_idx < csr_idx) == (B.avg() > oracle.break_even_avg(r, c))
    assert [oracle.break_even_avg(r, c) for r, c in [(1, 8), (2, 8), (4, 4), (4, 8), (8, 4)]] == [1.25, 1.5, 1.5, 2, 2]


def test_partition_rule_balances_blocks():
    A = inputs.rmat(12, seed=5)
    B = oracle.beta_convert(A, 2, 8)
    per_iv = np.diff(B.block_rowptr)
    for T in (1, 3, 16, 52):
        b = oracle.partition(B.block_rowptr, T)
        assert b[0] == 0 and b[-1] == len(per_iv) and np.all(np.diff(b) >= 0)
        loads = np.array([B.block_rowptr[b[t + 1]] - B.block_rowptr[b[t]] for t in range(T)])
        assert loads.sum() == B.nblocks
        # each boundary sits at the prefix nearest to its target
        for t in range(T - 1):
            target = (t + 1) * B.nblocks / T
            here = abs(target - B.block_rowptr[b[t + 1]])
            assert here <= abs(target - B.block_rowptr[min(b[t + 1] + 1, len(per_iv))]) + 1e-9
        assert np.all(np.abs(np.cumsum(loads)[:-1] - B.nblocks / T * np.arange(1, T)) <= per_iv.max() + 1)


def _partition_brute(brp, T):
    """Each boundary by exhaustion: from the previous boundary, the last interval
    index whose block prefix is nearest (exactly, in integers) to (t+1)*Nb/T."""
    brp = [int(v) for v in brp]
    I, nb = len(brp) - 1, brp[-1]
    b = [0]
    for t in range(T):
        if t == T - 1:
            b.append(I)
            continue
        d = [abs((t + 1) * nb - T * brp[i]) for i in range(b[-1], I + 1)]
        m = min(d)
        b.append(b[-1] + max(k for k, v in enumerate(d) if v == m))
    return b


def test_partition_equals_its_definition_by_exhaustion():
    rng = np.random.default_rng(9)
    cases = [np.array([0]), np.array([0, 0, 0]), np.array([0, 5]), np.array([0, 3, 3, 7, 9, 12])]
    for _ in range(300):
        I = int(rng.integers(0, 40))
        per = rng.integers(0, 6, I) * (rng.random(I) < 0.7)  # many empty intervals
        cases.append(np.concatenate([[0], np.cumsum(per)]))
    for brp in cases:
        for T in (1, 2, 3, 5, 8, 64):
            assert list(oracle.partition(brp, T)) == _partition_brute(brp, T), (list(brp), T)


def test_round_bf16_against_torch():
    torch = pytest.importorskip("torch")
    v = inputs.vec_normal(20000, seed=4) * 10.0 ** inputs.vec_uniform(20000, seed=5, lo=-3, hi=3)
    f32 = v.astype(np.float32)
    ours = oracle.round_bf16(f32.astype(np.float64))
    ref = torch.from_numpy(f32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert oracle.round_bf16(np.array([1.0 + 2.0**-8]))[0] == 1.0  # tie to even
    assert oracle.round_bf16(np.array([1.0 + 3 * 2.0**-8]))[0] == 1.0 + 2.0**-6


def test_dyadic_inputs_make_laplacian_spmv_exact():
    A = inputs.laplacian2d(128, 128)
    x = inputs.vec_dyadic(A.m, seed=0, bits=20)
    y = oracle.csr_spmv(A, x)
    yd, _ = oracle.csr_spmv_dot2(A, x)
    assert np.array_equal(y, yd)
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)  # exact in float32 too


# ------------------------------------------------------------------ SpMM

def test_spmm_oracle_against_dense_matmul_and_linearity():
    for seed, (n, m, k) in enumerate([(30, 40, 1), (17, 9, 4), (64, 64, 32)]):
        A = tiny_random(n, m, 0.2, 50 + seed)
        X = inputs.vec_uniform(m * k, seed=seed).reshape(m, k)
        D = A.to_dense()
        Y = oracle.csr_spmm(A, X)
        ref = np.array([[sum(D[i, q] * X[q, j] for q in range(m)) for j in range(k)] for i in range(n)])
        assert np.allclose(Y, ref, rtol=0, atol=1e-13 * (np.abs(D) @ np.abs(X)).max() + 1e-300)
        Yd, S = oracle.csr_spmm_dot2(A, X)
        assert np.all(np.abs(Yd - ref) <= 1e-14 * S + 1e-300)
        # column j equals the SpMV with column j
        assert np.array_equal(Y[:, 0], oracle.csr_spmv(A, np.ascontiguousarray(X[:, 0])))
        # linearity in X with exactly representable data
        X1 = inputs.vec_dyadic(m * k, seed=seed, bits=10).reshape(m, k)
        X2 = inputs.vec_dyadic(m * k, seed=seed + 7, bits=10).reshape(m, k)
        Ad = inputs.CSR(A.n, A.m, A.rowptr, A.colidx, inputs.vec_dyadic(A.nnz, seed=3, bits=10))
        assert np.array_equal(oracle.csr_spmm(Ad, X1 + X2), oracle.csr_spmm(Ad, X1) + oracle.csr_spmm(Ad, X2))


def test_poisson_shifted_is_symmetric_and_diagonally_dominant():
    A = inputs.poisson_shifted(5, 4, 3, seed=4)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.all(np.diag(D) > off)  # strictly dominant: positive definite
    assert np.all((np.diag(D) >= 6.0) & (np.diag(D) < 7.0))
    P = inputs.stencil3d(5, 4, 3, points=7, normal_values=False).to_dense()
    assert np.array_equal(D - np.diag(np.diag(D)), P - np.diag(np.diag(P)))
