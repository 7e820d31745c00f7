"""CPU oracle for block-shape selection.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Features (section "Performance prediction and optimal kernel selection":
  the average number of values per block, Avg(r,c) = N_nnz / N_blocks(r,c),
  can be had without converting the matrix; the paper's future-work section
  asks for more inputs such as statistics of the matrix): for the twelve
  shapes r in {1,2,4,8} x c in {4,8,16}, Avg(r,c); then the mean, standard
  deviation and maximum of the row lengths; then log10(n).
* The paper-style predictor (section "Performance polynomial interpolation"):
  per format, a least-squares polynomial of the performance in Avg(r,c);
  the format with the highest estimate is chosen.
* The paper's parallel predictor (same section, parallel part): per format a
  least-squares polynomial of the performance in two variables, Avg(r,c) and
  the amount of parallel hardware (the fraction of the SMs here), over the
  monomials Avg^a s^b with a + b <= degree; the highest estimate wins.
* A multilayer perceptron 16 (or 20) -> 64 -> 64 -> 12 with ReLU, in float64,
  that maps standardised features to a score per format (centred log time);
  its forward and backward passes written out layer by layer.
* Extended features (the conclusion's richer inputs): the 16 plus the mean
  distance |col - row| of the entries from the diagonal (over n, and as
  log10(1 + d)), the fraction of rows of at most two entries, and the
  fraction of the SMs used.
"""
from __future__ import annotations

import numpy as np

from . import SHAPES, beta_count

NFEAT = 16
NFMT = 12
HIDDEN = 64


def features(A) -> np.ndarray:
    """The 16 selection features of a CSR matrix."""
    f = np.zeros(NFEAT)
    for q, (r, c) in enumerate(SHAPES):
        nb = beta_count(A, r, c)[1]
        f[q] = A.nnz / nb if nb else 0.0
    lens = np.diff(np.asarray(A.rowptr, dtype=np.int64)).astype(np.float64)
    f[12] = lens.mean() if lens.size else 0.0
    f[13] = lens.std() if lens.size else 0.0
    f[14] = lens.max() if lens.size else 0.0
    f[15] = np.log10(max(A.n, 1))
    return f


def features_ext(A, sm_frac: float) -> np.ndarray:
    """The 20 extended features: the 16, then mean |col - row| / n,
    log10(1 + mean |col - row|), the fraction of rows with <= 2 entries, sm_frac."""
    f = np.zeros(20)
    f[:16] = features(A)
    rowptr = np.asarray(A.rowptr, dtype=np.int64)
    lens = np.diff(rowptr)
    rows = np.repeat(np.arange(A.n, dtype=np.int64), lens)
    dist = np.abs(np.asarray(A.colidx, dtype=np.int64) - rows)
    mean = float(dist.sum()) / A.nnz if A.nnz else 0.0
    f[16] = mean / A.n if A.n else 0.0
    f[17] = np.log10(1.0 + mean)
    f[18] = float((lens <= 2).sum()) / A.n if A.n else 0.0
    f[19] = sm_frac
    return f


# ---------------------------------------------------------------- polynomial

def poly_fit(avg: np.ndarray, perf: np.ndarray, degree: int) -> np.ndarray:
    """Least-squares coefficients c_0..c_d of perf ~ sum_j c_j avg^j."""
    V = np.vander(np.asarray(avg, dtype=np.float64), degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V, np.asarray(perf, dtype=np.float64), rcond=None)
    return coef


def poly_eval(coef: np.ndarray, avg) -> np.ndarray:
    return np.polynomial.polynomial.polyval(np.asarray(avg, dtype=np.float64), coef)


def poly_select(coefs: list[np.ndarray], feats: np.ndarray) -> int:
    """Index of the format with the highest estimated performance."""
    est = [poly_eval(coefs[q], feats[q]) for q in range(NFMT)]
    return int(np.argmax(est))


# ------------------------------------------------------------- 2D regression

def poly2_exponents(degree: int):
    """(a, b) of the monomials Avg^a s^b, a + b <= degree: by total degree, then by b."""
    return [(t - b, b) for t in range(degree + 1) for b in range(t + 1)]


def poly2_fit(avg: np.ndarray, sfrac: np.ndarray, perf: np.ndarray, degree: int) -> np.ndarray:
    """Least-squares coefficients of perf ~ sum_q c_q avg^a_q s^b_q for one format."""
    avg = np.asarray(avg, dtype=np.float64)
    sfrac = np.asarray(sfrac, dtype=np.float64)
    V = np.stack([avg**a * sfrac**b for a, b in poly2_exponents(degree)], axis=1)
    coef, *_ = np.linalg.lstsq(V, np.asarray(perf, dtype=np.float64), rcond=None)
    return coef


def poly2_eval(coef: np.ndarray, degree: int, avg, sfrac) -> np.ndarray:
    avg = np.asarray(avg, dtype=np.float64)
    return sum(c * avg**a * np.asarray(sfrac, dtype=np.float64)**b for c, (a, b) in zip(coef, poly2_exponents(degree)))


def poly2_select(coefs, degree: int, feats: np.ndarray, sfrac: float) -> int:
    """Index of the format with the highest 2D-regression estimate."""
    est = [poly2_eval(coefs[q], degree, feats[q], sfrac) for q in range(NFMT)]
    return int(np.argmax(est))


# ----------------------------------------------------------------------- MLP

def mlp_shapes(nfeat: int = NFEAT):
    return [(HIDDEN, nfeat), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (NFMT, HIDDEN), (NFMT,)]


def mlp_nparams(nfeat: int = NFEAT) -> int:
    return sum(int(np.prod(s)) for s in mlp_shapes(nfeat))


def mlp_unpack(theta: np.ndarray):
    """Split the flat parameter vector: W1, b1, W2, b2, W3, b3 (row-major); the
    input width follows from the vector's length."""
    nfeat = next(k for k in (NFEAT, 20) if mlp_nparams(k) == len(theta))
    out, o = [], 0
    for s in mlp_shapes(nfeat):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def mlp_forward(theta: np.ndarray, X: np.ndarray):
    """Scores (batch x 12) and the cached activations."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    out = H2 @ W3.T + b3
    return out, (X, Z1, H1, Z2, H2)


def mlp_loss(theta, X, Y, M=None):
    """Mean squared error over the (masked) outputs: sum(M (out - Y)^2) / sum(M)."""
    out, _ = mlp_forward(theta, X)
    M = np.ones_like(Y) if M is None else M
    return float((M * (out - Y) ** 2).sum() / M.sum())


def mlp_grad(theta, X, Y, M=None) -> np.ndarray:
    """Gradient of mlp_loss by the chain rule, layer by layer, flat like theta."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(theta)
    out, (X, Z1, H1, Z2, H2) = mlp_forward(theta, X)
    M = np.ones_like(Y) if M is None else M
    dOut = 2.0 * M * (out - Y) / M.sum()
    gW3 = dOut.T @ H2
    gb3 = dOut.sum(axis=0)
    dH2 = dOut @ W3
    dZ2 = dH2 * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    return np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), t >= 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**t)
    vh = v / (1 - b2**t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- targets

def centred_log_times(times: np.ndarray) -> np.ndarray:
    """Per matrix: log(t_f) minus the mean over formats (the score the MLP fits)."""
    lt = np.log(np.asarray(times, dtype=np.float64))
    return lt - lt.mean(axis=-1, keepdims=True)


def regret(times: np.ndarray, choice: np.ndarray) -> np.ndarray:
    """t(chosen) / t(best) - 1 per matrix."""
    times = np.asarray(times, dtype=np.float64)
    best = times.min(axis=1)
    return times[np.arange(times.shape[0]), choice] / best - 1.0
