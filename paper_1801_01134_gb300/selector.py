"""Block-shape selector: timing corpus, GPU-trained MLP and the paper-style
polynomial predictor, with regret on held-out matrices.

The paper predicts each kernel's performance from Avg(r,c) with one fitted
polynomial per kernel and takes the best estimate (section "Performance
prediction and optimal kernel selection"); its conclusion asks for richer
inputs. This module records SpMV timings of every block shape over generated
matrices with the library's own timing recorder (spc5_time_formats), trains
the library's MLP on the GPU (spc5_mlp_train) to score the shapes from the 16
features (spc5_features), fits the polynomial predictor (spc5_poly_fit) as the
fallback and yardstick, and reports the regret t(chosen) / t(best) - 1 of both on
held-out matrices. Timing, feature counting, MLP training and inference and
the polynomial fit run in libspc5; this module drives them and computes the
input standardisation and the regret statistics.

    python -m paper_1801_01134_gb300.selector --train 2000 --test 300 --out <file.npz>
"""
from __future__ import annotations

import argparse
import json
import queue
import threading
import time

import numpy as np
import torch

from . import inputs, spc5

SHAPES = spc5.SHAPES


def record(indices, seed: int = 3, dtype=torch.float64, reps: int = 5, n_max: float = 4e6, log=None):
    """Features, per-shape SpMV milliseconds and nnz for corpus matrices.

    Matrices are generated on the host by a producer thread (the generator
    releases the interpreter lock) while the GPU times the previous one."""
    q: "queue.Queue" = queue.Queue(maxsize=2)

    def produce():
        for i in indices:
            q.put((i, inputs.corpus_matrix(i, seed=seed, n_max=n_max)))
        q.put(None)

    th = threading.Thread(target=produce, daemon=True)
    th.start()
    F, T, NNZ, fam = [], [], [], []
    t0 = time.time()
    while True:
        item = q.get()
        if item is None:
            break
        i, A = item
        d = spc5.upload_csr(A, dtype, "cuda")
        F.append(spc5.features(d))
        T.append(spc5.time_formats(d, reps=reps))
        NNZ.append(A.nnz)
        fam.append(inputs.corpus_params(i, seed=seed, n_max=n_max)["family"])
        del d
        if log and len(F) % 100 == 0:
            log(f"recorded {len(F)} matrices in {time.time() - t0:.0f} s")
    th.join()
    return np.array(F), np.array(T, dtype=np.float64), np.array(NNZ, dtype=np.int64), fam


def mlp_inputs(F: np.ndarray, mean=None, scale=None):
    """x = (log1p(f) - mean) / scale, the input transform spc5_select applies."""
    L = np.log1p(np.asarray(F, dtype=np.float64))
    if mean is None:
        mean = L.mean(axis=0)
        scale = L.std(axis=0)
        # a constant feature (its spread only rounding noise) keeps a unit scale
        scale[scale <= 1e-9 * np.maximum(np.abs(mean), 1.0)] = 1.0
    return ((L - mean) / scale).astype(np.float32), mean.astype(np.float32), scale.astype(np.float32)


def centred_log(T: np.ndarray) -> np.ndarray:
    lt = np.log(T)
    return lt - lt.mean(axis=1, keepdims=True)


def regret(T: np.ndarray, choice) -> np.ndarray:
    choice = np.asarray(choice)
    return T[np.arange(T.shape[0]), choice] / T.min(axis=1) - 1.0


def train_mlp(F: np.ndarray, T: np.ndarray, epochs: int = 400, lr: float = 2e-3, seed: int = 0, batch: int = 32):
    X, mean, scale = mlp_inputs(F)
    Y = centred_log(T).astype(np.float32)
    M = np.ones_like(Y)
    g = torch.Generator().manual_seed(seed)
    # He initialisation for the ReLU layers, zero biases
    parts = []
    for fan_out, fan_in in ((64, 16), (64, 64), (12, 64)):
        parts.append(torch.randn(fan_out * fan_in, generator=g) * np.sqrt(2.0 / fan_in))
        parts.append(torch.zeros(fan_out))
    params = torch.cat(parts).float().cuda().contiguous()
    assert params.numel() == spc5.mlp_nparams()
    Xd, Yd, Md = (torch.from_numpy(a).cuda().contiguous() for a in (X, Y, M))
    hist = spc5.mlp_train(params, Xd, Yd, Md, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return params, mean, scale, hist


def mlp_choices(params: torch.Tensor, F: np.ndarray, mean, scale) -> np.ndarray:
    X, _, _ = mlp_inputs(F, mean, scale)
    S = spc5.mlp_infer(params, torch.from_numpy(X).cuda().contiguous()).cpu().numpy()
    return S.argmin(axis=1)


def fit_poly(F: np.ndarray, T: np.ndarray, nnz: np.ndarray, degree: int) -> np.ndarray:
    gflops = 2.0 * nnz[:, None] / (T * 1e-3) / 1e9
    return spc5.poly_fit(F[:, :12], gflops, degree)


def poly_choices(coef: np.ndarray, F: np.ndarray) -> np.ndarray:
    est = np.stack([np.polynomial.polynomial.polyval(F[:, q], coef[q]) for q in range(12)], axis=1)
    return est.argmax(axis=1)


def choose_poly_degree(F, T, nnz, degrees=(1, 2, 3, 4), folds: int = 5) -> int:
    """Degree with the lowest mean regret in k-fold cross-validation."""
    idx = np.arange(F.shape[0])
    best = None
    for deg in degrees:
        regs = []
        for k in range(folds):
            va = idx % folds == k
            tr = ~va
            if tr.sum() <= deg + 1:
                continue
            coef = fit_poly(F[tr], T[tr], nnz[tr], deg)
            regs.append(regret(T[va], poly_choices(coef, F[va])))
        m = float(np.concatenate(regs).mean()) if regs else np.inf
        if best is None or m < best[0]:
            best = (m, deg)
    return best[1]


def summary(r: np.ndarray) -> dict:
    return {"mean": float(r.mean()), "median": float(np.median(r)), "p90": float(np.quantile(r, 0.9)),
            "max": float(r.max()), "zero_regret_frac": float((r <= 1e-12).mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=300)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--n-max", type=float, default=4e6)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--out", default=None, help="npz with the corpus table, the models and the evaluation")
    args = ap.parse_args()
    spc5.load()
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    Ftr, Ttr, Ntr, famtr = record(range(args.train), args.seed, n_max=args.n_max, reps=args.reps, log=log)
    Fte, Tte, Nte, famte = record(range(args.train, args.train + args.test), args.seed, n_max=args.n_max,
                                  reps=args.reps, log=log)
    t_rec = time.time() - t0
    # model selection on a validation split of the training matrices: the
    # number of epochs and the seed with the lowest mean validation regret
    va = np.arange(Ftr.shape[0]) % 7 == 0
    best = None
    for ep in (50, 100, 200, 400, 800):
        for sd in (0, 1):
            p_, m_, s_, h_ = train_mlp(Ftr[~va], Ttr[~va], epochs=ep, seed=sd)
            rv = float(regret(Ttr[va], mlp_choices(p_, Ftr[va], m_, s_)).mean())
            log(f"epochs {ep} seed {sd}: validation mean regret {rv:.4f}")
            if best is None or rv < best[0]:
                best = (rv, ep, sd)
    params, mean, scale, hist = train_mlp(Ftr, Ttr, epochs=best[1], seed=best[2])
    deg = choose_poly_degree(Ftr, Ttr, Ntr)
    coef = fit_poly(Ftr, Ttr, Ntr, deg)
    r_mlp = regret(Tte, mlp_choices(params, Fte, mean, scale))
    r_poly = regret(Tte, poly_choices(coef, Fte))
    fixed = int(np.argmin(np.log(Ttr).mean(axis=0)))
    r_fixed = regret(Tte, np.full(Tte.shape[0], fixed))
    res = {"train": args.train, "test": args.test, "record_s": round(t_rec, 1), "poly_degree": deg,
           "mlp_epochs": best[1], "mlp_seed": best[2], "mlp_validation_regret": best[0],
           "mlp_final_loss": float(hist[-1]), "mlp_first_loss": float(hist[0]),
           "regret_mlp": summary(r_mlp), "regret_poly": summary(r_poly),
           "regret_fixed": {**summary(r_fixed), "shape": f"{SHAPES[fixed][0]}x{SHAPES[fixed][1]}"},
           "regret_mlp_train": summary(regret(Ttr, mlp_choices(params, Ftr, mean, scale)))}
    print(json.dumps(res), flush=True)
    if args.out:
        np.savez(args.out, Ftr=Ftr.astype(np.float32), Ttr=Ttr.astype(np.float32), Ntr=Ntr,
                 Fte=Fte.astype(np.float32), Tte=Tte.astype(np.float32), Nte=Nte, famtr=np.array(famtr),
                 famte=np.array(famte), mlp_params=params.cpu().numpy(), feat_mean=mean, feat_scale=scale,
                 poly_coef=coef, poly_degree=deg, loss_hist=hist, result=json.dumps(res))


if __name__ == "__main__":
    main()
