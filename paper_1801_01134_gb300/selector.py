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

The SM-count axis (the paper's parallel predictor, a 2D regression over the
thread count and Avg(r,c)): the timings are recorded again on SM-limited
streams (spc5_sm_stream_create) and the 2D regression (spc5_poly2_fit) is
fitted over (Avg(r,c), SM fraction); its held-out regret is reported per SM
count beside the SM-unaware predictors:

    python -m paper_1801_01134_gb300.selector --sm-counts 16,40,80,152 --train 400 --test 120 \
        --mlp-model <selector.npz> --out <sm.npz>
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


def record_sm(indices, sm_counts, seed: int = 3, dtype=torch.float64, reps: int = 5, n_max: float = 1e6, log=None):
    """Features, nnz, and per-SM-count per-shape SpMV milliseconds (N x S x 12):
    the timing recorder run on SM-limited streams."""
    streams = [spc5.SmStream(k) for k in sm_counts]
    got = [st.sms for st in streams]
    F, T, NNZ = [], [], []
    t0 = time.time()
    for i in indices:
        A = inputs.corpus_matrix(i, seed=seed, n_max=n_max)
        d = spc5.upload_csr(A, dtype, "cuda")
        F.append(spc5.features_ext(d, 1.0))  # the SM fraction (last input) is set per SM count later
        T.append([spc5.time_formats(d, reps=reps, stream=st.stream) for st in streams])
        NNZ.append(A.nnz)
        del d
        if log and len(F) % 100 == 0:
            log(f"recorded {len(F)} matrices x {len(streams)} SM counts in {time.time() - t0:.0f} s")
    for st in streams:
        st.destroy()
    return np.array(F), np.array(T, dtype=np.float64), np.array(NNZ, dtype=np.int64), got


def fit_poly2(F, T, nnz, sfrac, degree):
    """The paper's 2D regression over (Avg(r,c), SM fraction) on GFLOP/s, all SM counts pooled.
    T: N x S x 12, sfrac: S values."""
    N, S, _ = T.shape
    avg = np.repeat(F[:, None, :12], S, axis=1).reshape(N * S, 12)
    sf = np.tile(np.asarray(sfrac, dtype=np.float64), N)
    gflops = (2.0 * nnz[:, None, None] / (T * 1e-3) / 1e9).reshape(N * S, 12)
    return spc5.poly2_fit(avg, sf, gflops, degree)


def poly2_choices(coef, degree, F, sfrac_one: float) -> np.ndarray:
    return np.array([SHAPES.index(spc5.poly2_select(coef, degree, f, sfrac_one)[:2]) for f in F])


def ext_samples(F, T, sfrac):
    """(matrix, SM count) samples for the 20-input MLP: the extended features with
    the SM fraction as the last input, targets the centred log times."""
    N, S, _ = T.shape
    X = np.repeat(F[:, None, :], S, axis=1).copy()
    X[:, :, 19] = np.asarray(sfrac)[None, :]
    return X.reshape(N * S, 20), T.reshape(N * S, 12)


def train_mlp_ext(X, T, epochs: int, seed: int = 0, lr: float = 2e-3, batch: int = 32):
    Xn, mean, scale = mlp_inputs(X)
    Y = centred_log(T).astype(np.float32)
    g = torch.Generator().manual_seed(seed)
    parts = []
    for fan_out, fan_in in ((64, 20), (64, 64), (12, 64)):
        parts.append(torch.randn(fan_out * fan_in, generator=g) * np.sqrt(2.0 / fan_in))
        parts.append(torch.zeros(fan_out))
    params = torch.cat(parts).float().cuda().contiguous()
    assert params.numel() == spc5.mlp_nparams(20)
    Xd, Yd, Md = (torch.from_numpy(a).cuda().contiguous() for a in (Xn, Y, np.ones_like(Y)))
    hist = spc5.mlp_train(params, Xd, Yd, Md, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return params, mean, scale, hist


def sm_axis_main(args, log):
    """Record the SM-axis corpus, fit the 2D regression, report held-out regret per SM count."""
    sm_req = [int(v) for v in args.sm_counts.split(",")]
    Ftr, Ttr, Ntr, sms = record_sm(range(args.train), sm_req, args.seed, n_max=args.n_max, reps=args.reps, log=log)
    Fte, Tte, Nte, _ = record_sm(range(args.train, args.train + args.test), sm_req, args.seed, n_max=args.n_max,
                                 reps=args.reps, log=log)
    full = max(sms)
    sfrac = [k / full for k in sms]
    # degree of the 2D regression by cross-validation over the training matrices
    best = None
    idx = np.arange(Ftr.shape[0])
    for deg in (1, 2, 3):
        regs = []
        for k in range(5):
            va = idx % 5 == k
            coef = fit_poly2(Ftr[~va], Ttr[~va], Ntr[~va], sfrac, deg)
            for j, sf in enumerate(sfrac):
                regs.append(regret(Ttr[va, j], poly2_choices(coef, deg, Ftr[va], sf)))
        m = float(np.concatenate(regs).mean())
        if best is None or m < best[0]:
            best = (m, deg)
    deg2 = best[1]
    coef2 = fit_poly2(Ftr, Ttr, Ntr, sfrac, deg2)
    # SM-unaware yardsticks: the 1D polynomial fitted on the whole-GPU timings,
    # the committed whole-GPU MLP, the best single shape on the whole GPU
    jf = sms.index(full)
    deg1 = choose_poly_degree(Ftr, Ttr[:, jf], Ntr)
    coef1 = fit_poly(Ftr, Ttr[:, jf], Ntr, deg1)
    fixed = int(np.argmin(np.log(Ttr[:, jf]).mean(axis=0)))
    mlp = None
    if args.mlp_model:
        z = np.load(args.mlp_model)
        mlp = (torch.from_numpy(z["mlp_params"]).cuda(), z["feat_mean"], z["feat_scale"])
    # the MLP with the richer inputs (x-access locality, short rows, SM fraction),
    # epochs and seed chosen on a validation split of the training matrices
    va = np.arange(Ftr.shape[0]) % 7 == 0
    Xtr_v, Ttr_v = ext_samples(Ftr[~va], Ttr[~va], sfrac)
    best_m = None
    for ep in (50, 100, 200, 400):
        for sd in (0, 1):
            p_, m_, s_, _ = train_mlp_ext(Xtr_v, Ttr_v, ep, sd)
            rv = []
            for j, sf in enumerate(sfrac):
                Xv, _ = ext_samples(Ftr[va], Ttr[va][:, j:j + 1], [sf])
                rv.append(regret(Ttr[va, j], mlp_choices(p_, Xv, m_, s_)))
            rv = float(np.concatenate(rv).mean())
            log(f"extended MLP epochs {ep} seed {sd}: validation mean regret {rv:.4f}")
            if best_m is None or rv < best_m[0]:
                best_m = (rv, ep, sd)
    Xall, Tall = ext_samples(Ftr, Ttr, sfrac)
    pe, me, se, he = train_mlp_ext(Xall, Tall, best_m[1], best_m[2])
    per = {}
    for j, k in enumerate(sms):
        Xte_j, _ = ext_samples(Fte, Tte[:, j:j + 1], [sfrac[j]])
        row = {"sm_fraction": round(sfrac[j], 4),
               "mlp_ext": summary(regret(Tte[:, j], mlp_choices(pe, Xte_j, me, se))),
               "poly2": summary(regret(Tte[:, j], poly2_choices(coef2, deg2, Fte, sfrac[j]))),
               "poly_whole_gpu": summary(regret(Tte[:, j], poly_choices(coef1, Fte))),
               "fixed_whole_gpu": summary(regret(Tte[:, j], np.full(Tte.shape[0], fixed)))}
        if mlp is not None:
            row["mlp_whole_gpu"] = summary(regret(Tte[:, j], mlp_choices(mlp[0], Fte[:, :16], mlp[1], mlp[2])))
        # how often the best shape on k SMs differs from the best on the whole GPU
        row["best_differs_from_whole_gpu"] = float((Tte[:, j].argmin(axis=1) != Tte[:, jf].argmin(axis=1)).mean())
        per[str(k)] = row
    res = {"train": args.train, "test": args.test, "sm_counts": sms, "poly2_degree": deg2, "poly_degree": deg1,
           "mlp_ext_epochs": best_m[1], "mlp_ext_seed": best_m[2], "mlp_ext_validation_regret": best_m[0],
           "fixed_shape": f"{SHAPES[fixed][0]}x{SHAPES[fixed][1]}", "regret_by_sm_count": per}
    log(json.dumps(res))
    if args.out:
        np.savez(args.out, Ftr=Ftr.astype(np.float32), Ttr=Ttr.astype(np.float32), Ntr=Ntr,
                 Fte=Fte.astype(np.float32), Tte=Tte.astype(np.float32), Nte=Nte, sm_counts=np.array(sms),
                 poly2_coef=coef2, poly2_degree=deg2, mlp_ext_params=pe.cpu().numpy(), mlp_ext_mean=me,
                 mlp_ext_scale=se, mlp_ext_loss=he, result=json.dumps(res))


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
    ap.add_argument("--sm-counts", default=None, help="SM-count axis: comma list of SM counts (2D regression)")
    ap.add_argument("--mlp-model", default=None, help="SM-count axis: the whole-GPU model to evaluate beside it")
    args = ap.parse_args()
    spc5.load()
    log = lambda m: print(m, flush=True)  # noqa: E731
    if args.sm_counts:
        return sm_axis_main(args, log)
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
