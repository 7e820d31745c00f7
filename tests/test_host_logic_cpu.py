"""Host-side parts of the library that need no GPU, against the oracle: the
paper's per-format polynomial fit (Householder least squares in libspc5) and
the argument checks of the selection calls."""
import numpy as np
import pytest

from oracle import select as osel
from paper_1801_01134_gb300 import spc5


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_poly_fit_matches_oracle_on_the_host(deg):
    rng = np.random.default_rng(5 + deg)
    N = 40
    avg = rng.uniform(1, 30, (N, 12))
    perf = rng.uniform(10, 900, (N, 12))
    coef = spc5.poly_fit(avg, perf, deg)
    for q in range(12):
        ref = osel.poly_fit(avg[:, q], perf[:, q], deg)
        assert np.allclose(coef[q], ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


def test_poly_fit_recovers_an_exact_polynomial():
    # data lying on a known cubic per format: the fit returns its coefficients
    rng = np.random.default_rng(11)
    avg = rng.uniform(1, 16, (30, 12))
    true = rng.standard_normal((12, 4))
    perf = np.stack([np.polynomial.polynomial.polyval(avg[:, q], true[q]) for q in range(12)], axis=1)
    coef = spc5.poly_fit(avg, perf, 3)
    assert np.allclose(coef, true, rtol=1e-8, atol=1e-8)


def test_poly_fit_rejects_bad_arguments():
    avg = np.ones((3, 12))
    perf = np.ones((3, 12))
    with pytest.raises(spc5.Spc5Error) as ei:
        spc5.poly_fit(avg, perf, 7)  # more coefficients than the library fits
    assert ei.value.status == spc5.EINVAL


def test_selector_regret_and_targets():
    from paper_1801_01134_gb300 import selector

    rng = np.random.default_rng(3)
    T = rng.uniform(0.1, 2.0, (50, 12))
    best = T.argmin(axis=1)
    assert np.all(selector.regret(T, best) == 0.0)
    other = (best + 1) % 12
    r = selector.regret(T, other)
    assert np.allclose(r, T[np.arange(50), other] / T[np.arange(50), best] - 1.0) and np.all(r > 0)
    # training targets: log times centred per matrix (same ordering, rows sum to zero)
    Y = selector.centred_log(T)
    assert np.allclose(Y.sum(axis=1), 0.0) and np.array_equal(Y.argmin(axis=1), best)


def test_selector_input_transform_is_the_library_one():
    from paper_1801_01134_gb300 import selector

    rng = np.random.default_rng(4)
    F = rng.uniform(0.0, 50.0, (200, 16))
    F[:, 5] = 3.0  # a constant feature keeps a unit scale
    X, mean, scale = selector.mlp_inputs(F)
    assert np.allclose(X.mean(axis=0)[[0, 1, 2]], 0.0, atol=1e-5) and scale[5] == 1.0
    X2, _, _ = selector.mlp_inputs(F, mean, scale)  # the stored (float32) transform reapplied
    assert np.allclose(X, X2, atol=1e-5)
    assert np.allclose(X2, (np.log1p(F) - mean.astype(np.float64)) / scale.astype(np.float64), atol=1e-5)


def test_selector_poly_choices_match_the_oracle_rule():
    from paper_1801_01134_gb300 import selector

    rng = np.random.default_rng(6)
    coef = rng.standard_normal((12, 3))
    F = rng.uniform(1.0, 16.0, (40, 16))
    got = selector.poly_choices(coef, F)
    want = [osel.poly_select(list(coef), f) for f in F]
    assert list(got) == want


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


def test_partition_matches_the_oracle_and_its_definition():
    import oracle

    rng = np.random.default_rng(21)
    cases = [np.array([0]), np.array([0, 0, 0, 0]), np.array([0, 7]), np.array([0, 3, 3, 7, 9, 12])]
    for _ in range(300):
        I = int(rng.integers(0, 50))
        per = rng.integers(0, 9, I) * (rng.random(I) < 0.6)
        cases.append(np.concatenate([[0], np.cumsum(per)]).astype(np.int32))
    from paper_1801_01134_gb300 import inputs

    B = oracle.beta_convert(inputs.rmat(11, seed=3), 2, 8)  # power-law block counts
    cases.append(B.block_rowptr)
    for brp in cases:
        for T in (1, 2, 3, 7, 16, 100):
            got = spc5.partition(brp, T)
            assert list(got) == list(oracle.partition(brp, T)) == _partition_brute(brp, T), (T,)


def test_partition_rejects_bad_arguments():
    with pytest.raises(spc5.Spc5Error) as ei:
        spc5.partition(np.array([0, 1, 2]), 0)
    assert ei.value.status == spc5.EINVAL


def test_binding_checks_vectors_before_calling_the_library():
    import torch

    # a handle value that is never passed on: every call below fails in the binding first
    M = spc5.Matrix(0x10, n=10, m=7, nnz=0, r=1, c=4, vt=spc5.SPC5_F64)
    try:
        with pytest.raises(TypeError):
            M.spmv_acc(torch.zeros(7, dtype=torch.float32), torch.zeros(10, dtype=torch.float64))
        with pytest.raises(ValueError):
            M.spmv_acc(torch.zeros(6, dtype=torch.float64), torch.zeros(10, dtype=torch.float64))
        with pytest.raises(ValueError):
            M.spmv_noalloc(torch.zeros(7, dtype=torch.float64), torch.zeros(11, dtype=torch.float64))
        M32 = spc5.Matrix(0x10, n=4, m=4, nnz=0, r=2, c=8, vt=spc5.SPC5_BF16)
        try:
            assert M32.vector_dtype == torch.float32  # bfloat16 storage takes float32 vectors
            with pytest.raises(TypeError):
                M32.spmv_acc(torch.zeros(4, dtype=torch.bfloat16), torch.zeros(4, dtype=torch.float32))
        finally:
            M32._h = None
    finally:
        M._h = None  # never handed to spc5_destroy
    M._h = None
    with pytest.raises(ValueError):  # a destroyed matrix
        M.spmv_acc(torch.zeros(7, dtype=torch.float64), torch.zeros(10, dtype=torch.float64))


def test_library_poly2_fit_and_select_match_the_oracle():
    # the library's 2D regression (host code) against the oracle's, and its choice
    from oracle import select as osel
    from paper_1801_01134_gb300 import spc5

    rng = np.random.default_rng(7)
    N, deg = 80, 2
    avg = rng.uniform(1.0, 24.0, (N, 12))
    s = rng.choice([16 / 152, 40 / 152, 80 / 152, 1.0], N)
    perf = rng.uniform(50.0, 900.0, (N, 12))
    got = spc5.poly2_fit(avg, s, perf, deg)
    for q in range(12):
        want = osel.poly2_fit(avg[:, q], s, perf[:, q], deg)
        assert np.allclose(got[q], want, rtol=1e-9, atol=1e-9)
    for i in range(10):
        f = np.concatenate([avg[i], np.zeros(4)])
        r, c, est = spc5.poly2_select(got, deg, f, float(s[i]))
        q = osel.poly2_select(list(got), deg, f, float(s[i]))
        assert (r, c) == oracle_shapes()[q]


def oracle_shapes():
    import oracle

    return oracle.SHAPES


def test_committed_sm_axis_model_refits_and_its_axis_limits_the_gpu():
    # the committed SM-axis corpus: the stored 2D-regression coefficients come
    # back from the stored timings through the library's fit, and fewer SMs
    # make the larger products slower
    import json
    import os

    from paper_1801_01134_gb300 import selector, spc5

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1801_01134_gb300",
                        "models", "selector_sm_gb300.npz")
    z = np.load(path)
    sms = [int(v) for v in z["sm_counts"]]
    sf = [k / max(sms) for k in sms]
    deg = int(z["poly2_degree"])
    coef = selector.fit_poly2(z["Ftr"].astype(np.float64), z["Ttr"].astype(np.float64), z["Ntr"], sf, deg)
    assert np.allclose(coef, z["poly2_coef"], rtol=1e-6, atol=1e-6)
    T = z["Ttr"].astype(np.float64)
    big = z["Ntr"] > np.quantile(z["Ntr"], 0.75)
    assert np.median(T[big, 0].min(axis=1) / T[big, -1].min(axis=1)) > 2.0  # 16 SMs vs all
    res = json.loads(str(z["result"]))
    assert set(res["regret_by_sm_count"]) == {str(k) for k in sms}
