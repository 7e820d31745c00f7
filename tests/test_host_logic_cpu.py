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
