"""Pins of the selection oracle: features on matrices with known block
counts, exact polynomial recovery, and the MLP gradient against central
finite differences."""
import numpy as np

import oracle
from oracle import select as osel
from paper_1801_01134_gb300 import inputs


def test_features_known_matrices():
    # dense 64 x 64: every block full, Avg = r*c; rows all of length 64
    D = inputs.CSR.from_dense(np.ones((64, 64)))
    f = osel.features(D)
    assert list(f[:12]) == [r * c for r, c in oracle.SHAPES]
    assert f[12] == 64 and f[13] == 0 and f[14] == 64 and abs(f[15] - np.log10(64)) < 1e-15
    # identity: one value per block for every shape with r <= c
    I = inputs.CSR.from_dense(np.eye(64))
    f = osel.features(I)
    for q, (r, c) in enumerate(oracle.SHAPES):
        assert f[q] == (r if r <= c else c)
    # Laplacian 128x128, beta(1,8): 81408 / 48896 (hand-derived count)
    L = inputs.laplacian2d(128, 128)
    f = osel.features(L)
    assert f[oracle.SHAPES.index((1, 8))] == 81408 / 48896
    lens = np.diff(L.rowptr)
    assert f[12] == lens.mean() and f[14] == 5


def test_row_length_std_hand_worked():
    # row lengths 1, 1, 4 (and one more matrix with 0, 2, 4, 6): mean 2 and
    # population standard deviation sqrt(((1-2)^2 + (1-2)^2 + (4-2)^2) / 3) = sqrt(2);
    # for 0, 2, 4, 6: mean 3, sqrt((9 + 1 + 1 + 9) / 4) = sqrt(5)
    D = np.zeros((3, 8))
    D[0, 2] = 1.0
    D[1, 7] = 1.0
    D[2, :4] = 1.0
    f = osel.features(inputs.CSR.from_dense(D))
    assert f[12] == 2.0 and abs(f[13] - 2 ** 0.5) < 1e-15 and f[14] == 4.0
    E = np.zeros((4, 6))
    E[1, :2] = 1.0
    E[2, 1:5] = 1.0
    E[3, :] = 1.0
    f = osel.features(inputs.CSR.from_dense(E))
    assert f[12] == 3.0 and abs(f[13] - 5 ** 0.5) < 1e-15 and f[14] == 6.0


def test_poly_select_takes_the_highest_estimate():
    # the paper's predictor keeps the format whose polynomial promises the most
    # GFLOP/s at the matrix's Avg(r,c). Hand-built table: format q estimates
    # q + 1 at every Avg except format 7, whose estimate is 100 - Avg^2
    coefs = [np.array([q + 1.0]) for q in range(osel.NFMT)]
    coefs[7] = np.array([100.0, 0.0, -1.0])
    feats = np.zeros(osel.NFEAT)
    feats[:12] = 3.0  # estimate of format 7: 91, the highest
    assert osel.poly_select(coefs, feats) == 7
    feats[7] = 9.5  # 100 - 90.25 = 9.75 < 12: format 11 (estimate 12) is best
    assert osel.poly_select(coefs, feats) == 11
    # estimates that fall with Avg: the format with the smallest Avg wins
    coefs = [np.array([50.0, -2.0]) for _ in range(osel.NFMT)]
    feats[:12] = [5, 4, 9, 7, 2.5, 6, 8, 3, 11, 10, 12, 13]
    assert osel.poly_select(coefs, feats) == 4


def test_poly_fit_recovers_exact_polynomials():
    rng = np.random.default_rng(0)
    for deg in (1, 2, 3, 4):
        c = rng.standard_normal(deg + 1)
        x = np.linspace(1.0, 32.0, 40)
        y = np.polynomial.polynomial.polyval(x, c)
        got = osel.poly_fit(x, y, deg)
        assert np.allclose(got, c, rtol=1e-8, atol=1e-8)
        assert np.allclose(osel.poly_eval(got, x), y, rtol=1e-10, atol=1e-8)


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(osel.mlp_nparams()) * 0.3
    X = rng.standard_normal((7, osel.NFEAT))
    Y = rng.standard_normal((7, osel.NFMT))
    M = (rng.random((7, osel.NFMT)) > 0.2).astype(float)
    g = osel.mlp_grad(theta, X, Y, M)
    h = 1e-6
    idx = rng.choice(theta.size, 200, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (osel.mlp_loss(theta + e, X, Y, M) - osel.mlp_loss(theta - e, X, Y, M)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_forward_is_the_layer_composition():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(osel.mlp_nparams())
    X = rng.standard_normal((3, osel.NFEAT))
    W1, b1, W2, b2, W3, b3 = osel.mlp_unpack(theta)
    out, _ = osel.mlp_forward(theta, X)
    for s in range(3):
        h1 = [max(0.0, sum(W1[j, q] * X[s, q] for q in range(16)) + b1[j]) for j in range(64)]
        h2 = [max(0.0, sum(W2[j, q] * h1[q] for q in range(64)) + b2[j]) for j in range(64)]
        o = [sum(W3[j, q] * h2[q] for q in range(64)) + b3[j] for j in range(12)]
        assert np.allclose(out[s], o, rtol=1e-12, atol=1e-12)


def test_adam_minimises_a_quadratic_and_regret_definition():
    theta = np.array([3.0, -2.0])
    m = v = np.zeros(2)
    for t in range(1, 2001):
        theta, m, v = osel.adam_step(theta, 2 * theta, m, v, t, 0.05)
    assert np.all(np.abs(theta) < 1e-3)
    times = np.array([[1.0, 2.0, 4.0], [3.0, 1.5, 6.0]])
    assert np.allclose(osel.regret(times, np.array([0, 0])), [0.0, 1.0])
    c = osel.centred_log_times(times)
    assert np.allclose(c.sum(axis=1), 0.0)


def test_poly2_fit_recovers_exact_2d_polynomials():
    # data drawn from a known polynomial in (Avg, s): the fit returns it
    rng = np.random.default_rng(5)
    for deg in (1, 2, 3):
        terms = osel.poly2_exponents(deg)
        assert len(terms) == (deg + 1) * (deg + 2) // 2 and terms[:3] == [(0, 0), (1, 0), (0, 1)][:len(terms)]
        c = rng.standard_normal(len(terms))
        avg = rng.uniform(1.0, 20.0, 60)
        s = rng.choice([8 / 152, 40 / 152, 80 / 152, 1.0], 60)
        y = sum(ci * avg**a * s**b for ci, (a, b) in zip(c, terms))
        got = osel.poly2_fit(avg, s, y, deg)
        assert np.allclose(got, c, rtol=1e-7, atol=1e-7)


def test_poly2_select_takes_the_highest_estimate_at_the_sm_fraction():
    # format 3: 10 + 20 s (gains with SMs); format 5: 20 (flat); others 1.
    # At s = 0.25 the flat format wins (15 < 20), at s = 1 format 3 (30 > 20).
    deg = 1
    coefs = [np.array([1.0, 0.0, 0.0]) for _ in range(osel.NFMT)]
    coefs[3] = np.array([10.0, 0.0, 20.0])
    coefs[5] = np.array([20.0, 0.0, 0.0])
    f = np.full(osel.NFEAT, 2.0)
    assert osel.poly2_select(coefs, deg, f, 0.25) == 5
    assert osel.poly2_select(coefs, deg, f, 1.0) == 3


def test_features_ext_hand_worked():
    # rows: [0: cols 0, 3], [1: col 1], [2: cols 0, 2, 4, 5]; distances |col - row|:
    # 0, 3 | 0 | 2, 0, 2, 3 -> sum 10 over 7 entries; rows with <= 2 entries: 2 of 3
    D = np.zeros((3, 6))
    D[0, [0, 3]] = 1.0
    D[1, 1] = 1.0
    D[2, [0, 2, 4, 5]] = 1.0
    f = osel.features_ext(inputs.CSR.from_dense(D), 0.25)
    assert abs(f[16] - (10 / 7) / 3) < 1e-15 and abs(f[17] - np.log10(1 + 10 / 7)) < 1e-15
    assert abs(f[18] - 2 / 3) < 1e-15 and f[19] == 0.25
    assert np.array_equal(f[:16], osel.features(inputs.CSR.from_dense(D)))


def test_mlp_with_20_inputs_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    theta = rng.standard_normal(osel.mlp_nparams(20)) * 0.3
    X = rng.standard_normal((5, 20))
    Y = rng.standard_normal((5, osel.NFMT))
    g = osel.mlp_grad(theta, X, Y)
    h = 1e-6
    for i in rng.choice(theta.size, 80, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        fd = (osel.mlp_loss(theta + e, X, Y) - osel.mlp_loss(theta - e, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))
