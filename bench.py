"""SpMV throughput of the selected beta(r,c) format vs plain CSR on one GB300.

Workload: the four synthetic matrices shaped like the paper's benchmark set
(Table 1 stand-ins), values N(0,1) seed 1, x uniform[-1,1] seed 0:
  * 27-point 3D stencil on a 128^3 grid      n = 2,097,152   nnz = 55,742,968
  * FEM-like 3x3 dense blocks, 9-27 per block row, bandwidth 5%   n = 3,000,000
  * R-MAT scale 22, a/b/c = 0.57/0.19/0.19, 16 draws per vertex, relabelled
  * uniform random, n = 1,000,000, 8 entries per row
One step = one y = A x per matrix, each in the block shape picked for it by
exhaustive timing (the paper's "best kernel"), with the L2 cache flushed
before every product. value = sum(2 nnz) / sum(kernel time) in GFLOP/s
(the paper's 2 N_nnz / T).

Also reported on the same line: the plain CSR kernel on the same GPU, the
float32 form, an end-to-end figure with host buffers, the roofline of the
dominant kernel and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GFLOP/s & HBM GB/s (% of peak), selected β(r,c) vs CSR, 1 GB300"
L2_FLUSH_BYTES = 512 << 20
FP64_PEAK_GFLOPS = 1250.0  # nominal GB300 float64 rate (2 FMA lanes/clk/SM x 152 SMs x 2.07 GHz x 2)
# short-interval kernel variants the tuner tries per shape: float64 keeps to the
# flattened decodes (16's unrolled positions cost float64 pipe slots when empty)
VARIANTS = {"f64": (5, 10, 13, 15, 24), "f32": (5, 10, 13, 15, 16, 18, 24, 28)}
# beta(1,c) only: two lanes per row (natural, sorted order), Algorithm 2's single-value test (sorted, natural),
# the warp streaming its rows' blocks (float32 / bfloat16 only), two lanes per row with Algorithm 2's test
GROUP_VARIANTS = (22, 23, 30, 31, 32, 33)
CG_INNER_VARIANT = 18  # decode of the float32 / bfloat16 inner CG handle (unrolled positions, two blocks a trip)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--small", action="store_true", help="small matrices (quick functional run)")
    p.add_argument("--shapes", default="all", help="'all' or comma list like 1x8,2x4")
    p.add_argument("--profile", default=None,
                   help="profiling run: matrix name prefix (stencil27, fem3x3, rmat, uniform); runs --reps SpMVs")
    p.add_argument("--shape", default="4x8", help="block shape of the profiling run, e.g. 4x8, or csr")
    p.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"], help="profiling run value type")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--spmm-k", type=int, default=0, help="profiling run: time Y = A X with this many columns (float32)")
    p.add_argument("--ktile", type=int, default=0, help="profiling run: SpMM column tile (0 = from k)")
    p.add_argument("--variants", default="0", help="profiling run: comma list of kernel variants (0 = default)")
    p.add_argument("--order-window", type=int, default=0, help="profiling run: rows per work-order window "
                   "(0 = library default, negative = one window)")
    p.add_argument("--seg-blocks", type=int, default=0, help="profiling run: blocks per long-interval segment")
    p.add_argument("--long-blocks", type=int, default=0, help="profiling run: long-interval threshold in blocks")
    p.add_argument("--cg-profile", action="store_true", help="run the CG solvers once each with timings")
    p.add_argument("--unit-rates", action="store_true",
                   help="measure the float64 / float32 multiply-add rates (1..32 active lanes) and the copy ceiling")
    p.add_argument("--cg-n", type=int, default=96, help="grid edge of the CG profiling matrix")
    p.add_argument("--cg-every", type=int, default=8)
    p.add_argument("--cg-graph", type=int, default=1)
    p.add_argument("--cg-variant", type=int, default=18, help="kernel variant of the inner (float32) CG handle")
    p.add_argument("--cg-shape", default="2x4", help="block shape of the CG profiling handles")
    p.add_argument("--cg-inner-tol", type=float, default=0.0, help="inner tolerance of the mixed CG (0 = default)")
    return p.parse_args()


def workload(small: bool):
    from paper_1801_01134_gb300 import inputs

    if small:
        specs = [("stencil27_32^3", lambda: inputs.stencil3d(32, 32, 32, points=27, seed=1)),
                 ("fem3x3_n30k", lambda: inputs.block_fem(10000, seed=1)),
                 ("rmat_s14", lambda: inputs.rmat(14, seed=1)),
                 ("uniform_n100k", lambda: inputs.uniform(100000, 100000, 8, seed=1))]
    else:
        specs = [("stencil27_128^3", lambda: inputs.stencil3d(128, 128, 128, points=27, seed=1)),
                 ("fem3x3_n3M", lambda: inputs.block_fem(1000000, bs=3, bmin=9, bmax=27, band_frac=0.05, seed=1)),
                 ("rmat_s22", lambda: inputs.rmat(22, 16, 0.57, 0.19, 0.19, relabel=True, seed=1)),
                 ("uniform_n1M", lambda: inputs.uniform(1000000, 1000000, 8, seed=1))]
    return specs


def profile_matrices():
    """Mid-size members of the same families (above L2, a few hundred MB on the
    device) for hardware-counter captures."""
    from paper_1801_01134_gb300 import inputs

    return [("stencil27_96^3", lambda: inputs.stencil3d(96, 96, 96, points=27, seed=1)),
            ("fem3x3_n1M", lambda: inputs.block_fem(333334, bs=3, bmin=9, bmax=27, band_frac=0.05, seed=1)),
            ("rmat_s20", lambda: inputs.rmat(20, 16, 0.57, 0.19, 0.19, relabel=True, seed=1)),
            ("uniform_n1M", lambda: inputs.uniform(1000000, 1000000, 8, seed=1)),
            ("poisson7_96^3", lambda: inputs.stencil3d(96, 96, 96, points=7, normal_values=False))]


# sources that decide the SpMV kernels and the layout they read
SPMV_SOURCES = ("internal.cuh", "spmv_beta.cuh", "spmv_group.cuh", "spmv_stream.cuh", "spmv_f64.cu", "spmv_f32.cu",
                "spmv_bf16.cu", "spmv_group_f64.cu", "spmv_group_f32.cu", "spmv_group_bf16.cu", "convert.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1801_01134_gb300", "csrc")
    for f in SPMV_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_key(r: int, c: int, variant: int, dtype: str, workload_name: str) -> str:
    return f"beta({r},{c}) variant {variant} {dtype}|{workload_name}"


def profile_traffic(key: str):
    """DRAM bytes (read + write) of one SpMV from the committed ncu summary
    profiles/traffic.json, or None when the kernels changed since it was taken
    (the entry's source hash no longer matches)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    ent = rec.get("entries", {}).get(key)
    if not ent or rec.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_spmv")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


SLOWDOWN_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clocks: dict) -> bool:
    """True when the clock samples of a timed region saw a hardware or thermal
    slowdown (sw_power_cap alone is kept and noted)."""
    return any(r in SLOWDOWN_REASONS for r in clocks.get("reasons", []))


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v: float, ws: int, device=None) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ reference

def run_reference(args):
    """The CPU oracle (plain float64 CSR loop, OpenMP rows) on the same workload."""
    import oracle

    ws, rank, _ = dist_init(args)
    if rank != 0:
        return 0
    from paper_1801_01134_gb300 import inputs

    mats = [(name, gen()) for name, gen in workload(args.small)]
    xs = [inputs.vec_uniform(A.m, seed=0) for _, A in mats]
    flops = sum(2.0 * A.nnz for _, A in mats)
    for _ in range(args.warmup):
        for (_, A), x in zip(mats, xs):
            oracle.csr_spmv_omp(A, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for (_, A), x in zip(mats, xs):
            oracle.csr_spmv_omp(A, x)
    dt = time.perf_counter() - t0
    val = flops * args.steps / dt / 1e9
    threads = oracle.omp_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "suite4 float64: " + ", ".join(n for n, _ in mats), "format": "CSR (CPU oracle)",
                   "parallelism": "host OpenMP"},
        "cpu_baseline": {"value": round(val, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": f"full workload, {args.steps} steps of 4 CSR SpMVs, float64, {threads} threads"},
        "e2e": {"value": round(val, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ bytes, rooflines

VSIZE = {"f64": (8, 8), "f32": (4, 4), "bf16": (2, 4)}  # bytes per stored value, per x / y entry
NOMINAL_NOTE = "of nominal"


def beta_bytes(p, vsize, xsize):
    """Algorithmic bytes of one beta(r,c) SpMV: values + colidx + masks + block_rowptr
    + valptr + x + y, x counted once."""
    A, r, c = p["A"], p["r"], p["c"]
    I = (A.n + r - 1) // r
    mb = (r * c + 7) // 8
    return vsize * A.nnz + (4 + mb) * p["nblocks"] + 4 * (I + 1) + 8 * (I + 1) + xsize * A.m + xsize * A.n


def csr_bytes(p, vsize, xsize):
    """Algorithmic bytes of one CSR SpMV (int64 row pointer here)."""
    A = p["A"]
    return vsize * A.nnz + 4 * A.nnz + 8 * (A.n + 1) + xsize * A.m + xsize * A.n


def measured_hbm_peak():
    """The measured copy ceiling (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), \
            "MEASURED_PEAKS.json hbm_gbs: copy ceiling (of measured)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def spmv_kernel_names(p):
    """The kernels one product of a prepared matrix launches (names as ncu lists them)."""
    v, fused = p["variant"], p["nseg"] > 0 and p["variant"] != 1
    if v in (22, 23):
        rows, both = "k_spmv_rows_g", "k_spmv_rows_segs"
    elif v == 33:
        rows, both = "k_spmv_rows_g1", "k_spmv_g1_segs"
    elif v in (30, 31):
        rows, both = "k_spmv_rows_t", "k_spmv_t_segs"
    elif v == 32:
        rows, both = "k_spmv_s", "k_spmv_s_segs"
    elif 24 <= v <= 29:
        rows, both = "k_spmv_grp", "k_spmv_grp_segs"
    elif v == 1:
        rows, both = "k_spmv_rows", None
    else:
        rows, both = "k_spmv_rows_u", "k_spmv_rows_segs"
    if p["nseg"] > 0:
        return (both if fused else f"{rows}+k_spmv_segments") + "+k_spmv_fixup"
    return rows


def roofline_entry(p, tlist, key, hbm_peak, hbm_src, hbm_nominal):
    """HBM roofline of one matrix's product: algorithmic bytes / mean duration."""
    t = statistics.mean(tlist)
    b = beta_bytes(p, *VSIZE[key])
    gbs = b / t / 1e6
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
            "traffic": profile_traffic(traffic_key(p["r"], p["c"], p["variant"], key, p["name"])),
            "algorithmic_bytes": int(b), "mean_ms": round(t, 4),
            "kernel": f"{spmv_kernel_names(p)}<{p['r']},{p['c']},{key}> variant {p['variant']} on {p['name']}",
            "peak_source": hbm_src, "nominal_peak": round(hbm_nominal, 1),
            "frac_of_nominal": round(gbs / hbm_nominal, 4)}


def matrix_entry(p, tlist, key, hbm_peak, roofline=None):
    t = statistics.median(tlist)
    A = p["A"]
    gbs = beta_bytes(p, *VSIZE[key]) / t / 1e6
    e = {"matrix": p["name"], "n": A.n, "nnz": A.nnz, "shape": f"{p['r']}x{p['c']}", "variant": p["variant"],
         "convert_ms": round(p["convert_ms"], 3), "convert_over_spmv": round(p["convert_ms"] / t, 2),
         "avg_nnz_per_block": round(A.nnz / max(p["nblocks"], 1), 3), "segments": p["nseg"], "ms": round(t, 4),
         "gflops": round(2.0 * A.nnz / t / 1e6, 1), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
         "sweep_gflops": p["sweep_gflops"]}
    if roofline is not None:
        e["roofline"] = roofline
    return e


# ---------------------------------------------------------------------- SpMM

def precision_errors(prep, y64_ref):
    """Error of a float32 or bfloat16 storage form against the float64 product of the
    same matrix and x (the float64 result the tests hold to the oracle within
    1e-13 (|A||x|)_i), per matrix: max_i |y_i - y64_i| / max_i |y64_i| and the
    relative 2-norm; x is the float32 rounding of the float64 x."""
    import torch

    def measures(y, y64):
        d = (y.double() - y64).abs()
        return {"max_rel_to_max": float(d.max() / y64.abs().max().clamp_min(1e-300)),
                "rel_l2": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(y64).clamp_min(1e-300))}

    out = {}
    try:
        for p in prep:
            out[p["name"]] = {"shape": f"{p['r']}x{p['c']}", **measures(p["M"].spmv(p["x"]), y64_ref[p["name"]])}
    except Exception as e:  # reporting only: never costs the measured line
        out["unavailable"] = f"{type(e).__name__}: {e}"
    return out


def run_spmm_section(mats, dev, ks=(1, 4, 8, 16, 32), reps: int = 5):
    """float32 Y = A X for k right-hand sides on the stencil and R-MAT matrices, in the
    (shape, column tile) the library's tuner picks per k (spc5_tune); GFLOP/s = 2 nnz k / t,
    HBM fraction with X and Y counted k-fold."""
    import torch

    from paper_1801_01134_gb300 import spc5

    fa = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    fb = torch.empty_like(fa)
    hbm_peak, _ = measured_hbm_peak()

    def timed(fn):
        ts = []
        for _ in range(reps):
            spc5.copy(fa, fb)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:]) if len(ts) > 1 else ts[0]

    out = {}
    for mt in mats:
        if not (mt["name"].startswith("stencil") or mt["name"].startswith("rmat")):
            continue
        A = mt["A"]
        d = spc5.upload_csr(A, torch.float32, dev)
        res = {}
        for k in ks:
            tn = spc5.tune(d, k_spmm=k, reps=3)
            M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, tn["spmm_r"], tn["spmm_c"],
                             variant=tn["spmm_variant"])
            X = torch.rand(A.m, k, dtype=torch.float32, device=dev)
            Y = torch.empty(A.n, k, dtype=torch.float32, device=dev)
            t = timed(lambda: M.spmm(X, Y, ktile=tn["ktile"]))
            p = {"A": A, "r": tn["spmm_r"], "c": tn["spmm_c"], "nblocks": M.export()["nblocks"]}
            r, c = tn["spmm_r"], tn["spmm_c"]
            I = (A.n + r - 1) // r
            nbytes = 4 * A.nnz + (4 + (r * c + 7) // 8) * p["nblocks"] + 12 * (I + 1) + 4 * k * (A.m + A.n)
            res[f"k{k}"] = {"ms": round(t, 4), "gflops": round(2.0 * A.nnz * k / t / 1e6, 1),
                            "shape": f"{r}x{c}", "ktile": tn["ktile"], "gbs": round(nbytes / t / 1e6, 1),
                            "hbm_frac": round(nbytes / t / 1e6 / hbm_peak, 4)}
            M.destroy()
            del X, Y
        out[mt["name"]] = res
        del d
    return out


# ------------------------------------------------------------------ selector

def run_selector_section(prep, dev):
    """Shapes the committed MLP and polynomial models pick for the bench
    matrices, with their regret against the exhaustive sweep of the run, and
    the models' held-out regret from the corpus they were trained on."""
    import numpy as np

    from paper_1801_01134_gb300 import spc5

    path = os.path.join(ROOT, "paper_1801_01134_gb300", "models", "selector_gb300.npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    import torch

    P = torch.from_numpy(z["mlp_params"]).to(dev)
    out = {"model": "paper_1801_01134_gb300/models/selector_gb300.npz",
           "held_out": {k: json.loads(str(z["result"]))[k] for k in ("regret_mlp", "regret_poly", "regret_fixed")}}
    per = {}
    for p in prep:
        d = p["d"]
        sweep = p["sweep_gflops"]
        best = max(sweep.values())
        rm, cm, _ = spc5.select(d, spc5.SELECT_MLP, mlp_params=P, feat_mean=z["feat_mean"], feat_scale=z["feat_scale"])
        rp, cp, _ = spc5.select(d, spc5.SELECT_POLY, poly_coef=z["poly_coef"])
        per[p["name"]] = {"best": f"{p['r']}x{p['c']}", "mlp": f"{rm}x{cm}",
                          "mlp_regret": round(best / sweep[f"{rm}x{cm}"] - 1.0, 4),
                          "poly": f"{rp}x{cp}", "poly_regret": round(best / sweep[f"{rp}x{cp}"] - 1.0, 4)}
    out["bench_matrices"] = per
    smp = os.path.join(ROOT, "paper_1801_01134_gb300", "models", "selector_sm_gb300.npz")
    if os.path.exists(smp):
        zs = np.load(smp)
        rs = json.loads(str(zs["result"]))
        out["sm_axis"] = {"model": "paper_1801_01134_gb300/models/selector_sm_gb300.npz",
                          "what": "held-out mean regret per SM count (green-context partitions): the paper's 2D "
                                  "regression over (Avg, SM fraction) beside the SM-unaware whole-GPU predictors",
                          "poly2_degree": rs["poly2_degree"],
                          "mean_regret": {k: {m: round(v[m]["mean"], 4) for m in v if isinstance(v[m], dict)}
                                          for k, v in rs["regret_by_sm_count"].items()},
                          "best_differs_from_whole_gpu": {k: v["best_differs_from_whole_gpu"]
                                                          for k, v in rs["regret_by_sm_count"].items()}}
    return out


# ------------------------------------------------------------------- batched

def run_batch_section(dev, count: int = 256, reps: int = 20):
    """256 uneven float32 matrices (n lognormal in [1k, 64k], 3..60 per row,
    stencil / banded / uniform, seed 2), each in the shape and kernel variant the
    library's tuner picks for it (spc5_tune): one graph-replayed persistent launch vs
    one SpMV launch per matrix. GFLOP/s = sum(2 nnz) / t."""
    import torch

    from paper_1801_01134_gb300 import inputs, spc5

    mats, keep, xs, ys, shapes, variants = [], [], [], [], {}, {}
    flops = 0.0
    nbytes = 0
    t_tune = time.time()
    for j in range(count):
        A = inputs.batch_matrix(j, seed=2)
        d = spc5.upload_csr(A, torch.float32, dev)
        tn = spc5.tune(d, reps=3)
        r, c, v = tn["r"], tn["c"], tn["variant"]
        shapes[f"{r}x{c}"] = shapes.get(f"{r}x{c}", 0) + 1
        variants[str(v)] = variants.get(str(v), 0) + 1
        M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=v)
        mats.append(M)
        nbytes += beta_bytes({"A": A, "r": r, "c": c, "nblocks": M.export()["nblocks"]}, 4, 4)
        keep.append(d)
        xs.append(torch.rand(A.m, dtype=torch.float32, device=dev))
        ys.append(torch.empty(A.n, dtype=torch.float32, device=dev))
        flops += 2.0 * A.nnz
    t_tune = time.time() - t_tune
    B = spc5.Batch(mats, xs, ys)

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    t_graph = timed(lambda: B.run(graph=True))
    t_direct = timed(lambda: B.run(graph=False))

    def each():
        for M, x, y in zip(mats, xs, ys):
            M.spmv(x, y)

    t_each = timed(each)
    B.destroy()
    for M in mats:
        M.destroy()
    hbm_peak, _ = measured_hbm_peak()
    return {"workload": f"{count} float32 matrices, n lognormal in [1k, 64k], 3..60 per row, seed 2",
            "nnz_total": int(flops / 2), "shapes": shapes, "variants": variants, "tune_s": round(t_tune, 2),
            "tuner": "spc5_tune per matrix (shape x variant, timed, cached per signature)",
            "graph_ms": round(t_graph, 4), "gflops_graph": round(flops / t_graph / 1e6, 1),
            "gbs_graph": round(nbytes / t_graph / 1e6, 1), "hbm_frac_graph": round(nbytes / t_graph / 1e6 / hbm_peak, 4),
            "direct_ms": round(t_direct, 4), "gflops_direct": round(flops / t_direct / 1e6, 1),
            "per_matrix_launches_ms": round(t_each, 4), "gflops_per_matrix_launches": round(flops / t_each / 1e6, 1),
            "speedup_vs_per_matrix": round(t_each / t_graph, 3),
            "l2": "not flushed between replays (the batch's arrays, ~0.5 GB, exceed L2)"}


# ------------------------------------------------------------------------ CG

def run_cg_section(dev, reps: int = 3, shifted: bool = False):
    """Time float64 CG and mixed float32 / bfloat16 refinement to ||r|| / ||b|| <= 1e-10
    on the 7-point Poisson matrix of a 96^3 grid (b uniform[-1,1] seed 0). Its values
    6 / -1 are exact in float32 and bfloat16, so the low-precision inner matrices equal
    the float64 one there; with shifted=True the diagonal is raised by a seeded uniform
    [0, 1) draw per row, and the inner matrices are rounded copies."""
    import torch

    from paper_1801_01134_gb300 import inputs, spc5

    A = inputs.poisson_shifted(96, 96, 96, seed=4) if shifted else \
        inputs.stencil3d(96, 96, 96, points=7, normal_values=False)
    b = torch.from_numpy(inputs.vec_uniform(A.n, seed=0)).to(dev)
    hs = {}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32), ("bf16", torch.bfloat16)):
        d = spc5.upload_csr(A, dt, dev)
        hs[name] = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 4,
                                variant=0 if name == "f64" else CG_INNER_VARIANT)
    out = {"workload": ("7-point Poisson 96^3, diagonal 6 + uniform[0,1) seed 4 (values round in bf16 / f32)" if shifted
                        else "7-point Poisson 96^3 (values 6 / -1, exact in bf16 and f32)") +
                       " (n=884,736, nnz=6,137,856), b uniform[-1,1] seed 0, tol 1e-10",
           "format": f"beta(2,4); float64 handle variant 5, inner handles variant {CG_INNER_VARIANT}"}
    for label, inner, rel in (("fp64_cg", None, False), ("mixed_f32", hs["f32"], False),
                              ("mixed_bf16", hs["bf16"], False), ("reliable_f32", hs["f32"], True),
                              ("reliable_bf16", hs["bf16"], True)):
        ts, info = [], None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x, info = spc5.cg(hs["f64"], b, A_inner=inner, tol=1e-10, use_graph=True, reliable=rel)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[label] = {"ms": round(min(ts), 3), "iterations": info["iterations"], "outer": info["outer"],
                      "rel_residual": info["rel_residual"], "converged": info["converged"]}
    for k in ("mixed_f32", "mixed_bf16", "reliable_f32", "reliable_bf16"):
        out[f"speedup_{k}"] = round(out["fp64_cg"]["ms"] / out[k]["ms"], 3)
    for h in hs.values():
        h.destroy()
    return out


# ---------------------------------------------------------------- CPU baseline

def run_cpu_baseline(mats, prep64, budget_s: float = 20.0):
    """The oracle as it stands on the host cores, timed as the paper times its kernels
    (mean of 16 runs): the plain CSR loop over all cores (the reported value) and on one
    core, and the oracle's product read from the beta(r,c) arrays (one core) in each
    matrix's selected shape. Run counts shrink so that the whole sample stays near
    budget_s seconds of CPU time."""
    import oracle

    flops = sum(2.0 * mt["A"].nnz for mt in mats)

    def mean_runs(fn, runs):
        ts = []
        for _ in range(runs):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.mean(ts), runs

    def suite(f):
        for mt in mats:
            f(mt["A"], mt["x"])

    t_all, n_all = mean_runs(lambda: suite(oracle.csr_spmv_omp), 16)
    t1 = mean_runs(lambda: suite(oracle.csr_spmv), 1)[0]
    t_one, n_one = mean_runs(lambda: suite(oracle.csr_spmv), max(1, min(16, int(budget_s * 0.5 / max(t1, 1e-9)))))
    beta = {}
    shapes = {p["name"]: (p["r"], p["c"]) for p in prep64}
    for mt in mats:
        A = mt["A"]
        r, c = shapes[mt["name"]]
        B = oracle.beta_convert(A, r, c)
        tb1 = mean_runs(lambda: oracle.beta_spmv(B, mt["x"]), 1)[0]
        tb, nb = mean_runs(lambda: oracle.beta_spmv(B, mt["x"]), max(1, min(16, int(budget_s * 0.1 / max(tb1, 1e-9)))))
        beta[mt["name"]] = {"shape": f"{r}x{c}", "gflops": round(2.0 * A.nnz / tb / 1e9, 3), "runs": nb}
        del B
    cores = oracle.omp_threads()
    return {"value": round(flops / t_all / 1e9, 3), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"mean of {n_all} runs of the 4 float64 CSR SpMVs (plain loop, OpenMP over rows, "
                      f"{cores} threads), full matrices",
            "single_thread": {"value": round(flops / t_one / 1e9, 3), "unit": "GFLOP/s", "runs": n_one,
                              "sample": "the same loop on one core"},
            "beta_oracle_one_core": beta}


# ------------------------------------------------------------------ profiling

def run_profile(args):
    """One matrix, one format: convert, then --reps SpMVs with an L2 flush before
    each (the command line that the ncu summaries under profiles/ quote)."""
    import torch

    from paper_1801_01134_gb300 import inputs, spc5

    spc5.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    name, gen = next((n, g) for n, g in workload(args.small) + profile_matrices() if n.startswith(args.profile))
    A = gen()
    vdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[args.dtype]
    xdt = torch.float64 if args.dtype == "f64" else torch.float32
    d = spc5.upload_csr(A, vdt, dev)
    x = torch.from_numpy(inputs.vec_uniform(A.m, seed=0)).to(dev).to(xdt)
    y = torch.empty(A.n, dtype=xdt, device=dev)
    fa = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    fb = torch.empty_like(fa)
    for shape in args.shape.split(","):
        for variant in (int(v) for v in args.variants.split(",")):
            if shape == "csr":
                run = lambda: spc5.csr_spmv(d.rowptr, d.colidx, d.values, A.n, A.m, x, y, group=variant)  # noqa: E731
                fmt = f"csr group={variant}"
            else:
                r, c = (int(v) for v in shape.split("x"))
                M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=variant,
                                 order_window=args.order_window, seg_blocks=args.seg_blocks,
                                 long_blocks=args.long_blocks)
                run = lambda: M.spmv(x, y)  # noqa: E731
                ar = M.arrays()
                fmt = (f"beta({r},{c}) variant={variant} nblocks={ar.nblocks} segments={ar.nsegments}"
                       f" order_window={args.order_window} seg_blocks={args.seg_blocks} long_blocks={args.long_blocks}")
                if args.spmm_k > 0:  # Y = A X with spmm_k columns instead
                    X = torch.rand(A.m, args.spmm_k, dtype=xdt, device=dev)
                    Y = torch.empty(A.n, args.spmm_k, dtype=xdt, device=dev)
                    run = lambda: M.spmm(X, Y, ktile=args.ktile)  # noqa: E731
                    fmt += f" spmm k={args.spmm_k} ktile={args.ktile}"
            ts = []
            for _ in range(args.reps):
                spc5.copy(fa, fb)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                run()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            best = min(ts)
            kk = args.spmm_k if args.spmm_k > 0 and shape != "csr" else 1
            print(json.dumps({"profile": name, "format": fmt, "dtype": args.dtype, "n": A.n, "nnz": A.nnz,
                              "ms": [round(t, 4) for t in ts], "gflops_best": round(2.0 * A.nnz * kk / best / 1e6, 1)}),
                  flush=True)
            if shape != "csr":
                M.destroy()
    return 0


def run_unit_rates():
    """Arithmetic and copy rates of this GPU through the library's probe kernels:
    multiply-add rate with 1, 8, 16 and 32 active lanes per warp (only active
    lanes' FMAs counted), and the streaming copy (read + write bytes)."""
    import torch

    from paper_1801_01134_gb300 import spc5

    spc5.load()
    out = {"gpu": torch.cuda.get_device_name(0)}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        out[f"fma_{name}_gflops"] = {str(ln): round(spc5.fma_rate(dt, lanes=ln), 1) for ln in (1, 8, 16, 32)}
    n = 1 << 28  # 1 GiB of int32 per buffer
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    ts = []
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        spc5.copy(a, b)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    out["copy_gbs"] = round(2 * 4 * n / (min(ts[1:]) * 1e-3) / 1e9, 1)
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------ ours

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    if args.unit_rates:
        return run_unit_rates()
    if args.cg_profile:
        import torch

        from paper_1801_01134_gb300 import inputs, spc5

        spc5.load()
        dev = torch.device("cuda", 0)
        N = args.cg_n
        A = inputs.stencil3d(N, N, N, points=7, normal_values=False)
        b = torch.from_numpy(inputs.vec_uniform(A.n, seed=0)).to(dev)
        hs = {}
        for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
            d = spc5.upload_csr(A, dt, dev)
            r, c = (int(v) for v in args.cg_shape.split("x"))
            # --cg-variant sets the inner (float32) handle; the float64 handle keeps the default
            hs[name] = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c,
                                    variant=0 if name == "f64" else args.cg_variant)
        for label, inner, rel in (("fp64_cg", None, False), ("mixed_f32", hs["f32"], False),
                                  ("reliable_f32", hs["f32"], True)):
            for rep in range(2):
                t0 = time.perf_counter()
                x, info = spc5.cg(hs["f64"], b, A_inner=inner, tol=1e-10, check_every=args.cg_every,
                                  use_graph=bool(args.cg_graph), inner_tol=args.cg_inner_tol, reliable=rel)
                dt = time.perf_counter() - t0
                print(json.dumps({"solver": label, "rep": rep, "ms": round(dt * 1e3, 3), **info}), flush=True)
        return 0
    import torch

    from paper_1801_01134_gb300 import inputs, spc5

    ws, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    spc5.load()
    shapes = spc5.SHAPES if args.shapes == "all" else [tuple(int(v) for v in s.split("x")) for s in args.shapes.split(",")]

    # inputs: host generation, one upload (outside every timed region)
    mats = []
    for name, gen in workload(args.small):
        A = gen()
        x = inputs.vec_uniform(A.m, seed=0)
        mats.append({"name": name, "A": A, "x": x})
    flush_a = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_b = torch.empty_like(flush_a)

    def flush():
        spc5.copy(flush_a, flush_b)

    def time_call(fn, reps, warm=2):
        for _ in range(warm):
            flush()
            fn()
        ts = []
        for _ in range(reps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def prepare(dtype):
        """Upload, time every shape (exhaustive selection) and the CSR variants."""
        xdt = torch.float64 if dtype == torch.float64 else torch.float32
        out = []
        for mt in mats:
            A = mt["A"]
            d = spc5.upload_csr(A, dtype, dev)
            xd = torch.from_numpy(mt["x"]).to(dev).to(xdt)
            yd = torch.empty(A.n, dtype=xdt, device=dev)
            best = None
            sweep = {}
            for (r, c) in shapes:
                M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c)
                tv = {}
                group = tuple(v for v in GROUP_VARIANTS if dtype != torch.float64 or v != 32)
                for v in VARIANTS["f64" if dtype == torch.float64 else "f32"] + (group if r == 1 else ()):
                    M.set_variant(v)
                    tv[v] = time_call(lambda: M.spmv(xd, yd), 5)
                v = min(tv, key=tv.get)
                t = tv[v]
                M.set_variant(v)
                sweep[f"{r}x{c}"] = round(2.0 * A.nnz / t / 1e6, 1)
                if best is None or t < best[0]:
                    if best is not None:
                        best[1].destroy()
                    best = (t, M, r, c, v)
                else:
                    M.destroy()
            # the CSR comparator: plain (G lanes per row) and with long rows split into
            # warp segments like the β path (CsrPlan); the fastest is kept
            csr_best, csr_plain = None, None
            for g in (1, 2, 4, 8, 16, 32):
                t = time_call(lambda: spc5.csr_spmv(d.rowptr, d.colidx, d.values, A.n, A.m, xd, yd, group=g), 5)
                if csr_plain is None or t < csr_plain[0]:
                    csr_plain = (t, g)
                P = spc5.CsrPlan(d, group=g)
                if P.nsegments > 0:
                    tp = time_call(lambda: P.spmv(xd, yd), 5)
                    if csr_best is None or tp < csr_best[0]:
                        if csr_best is not None and csr_best[2] is not None:
                            csr_best[2].destroy()
                        csr_best = (tp, g, P)
                        continue
                P.destroy()
            if csr_best is None or csr_plain[0] <= csr_best[0]:
                if csr_best is not None:
                    csr_best[2].destroy()
                csr_best = (csr_plain[0], csr_plain[1], None)
            _, M, r, c, v = best
            ex = M.export()
            # conversion cost of the selected form (wall clock of spc5_convert, best of 3)
            conv = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                M2 = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, r, c, variant=v)
                torch.cuda.synchronize()
                conv.append((time.perf_counter() - t0) * 1e3)
                M2.destroy()
            out.append({"name": mt["name"], "A": A, "d": d, "x": xd, "y": yd, "M": M, "r": r, "c": c, "variant": v,
                        "nblocks": ex["nblocks"], "nseg": ex["nsegments"], "csr_group": csr_best[1],
                        "csr_plan": csr_best[2], "csr_plain_ms": csr_plain[0],
                        "sweep_gflops": sweep, "convert_ms": min(conv)})
        return out

    def run_steps(prep, K, W, fn_name="beta", sampler=None):
        per = {p["name"]: [] for p in prep}
        for step in range(W + K):
            for p in prep:
                flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if fn_name == "beta":
                    p["M"].spmv(p["x"], p["y"])
                elif p["csr_plan"] is not None:
                    p["csr_plan"].spmv(p["x"], p["y"])
                else:
                    A, d = p["A"], p["d"]
                    spc5.csr_spmv(d.rowptr, d.colidx, d.values, A.n, A.m, p["x"], p["y"], group=p["csr_group"])
                e1.record(stream)
                if step >= W:
                    per[p["name"]].append((e0, e1))
        torch.cuda.synchronize()
        return {k: [a.elapsed_time(b) for a, b in v] for k, v in per.items()}

    def csr_section(prep, K, key, beta_value, beta_times):
        """The CSR comparator (lanes per row tuned per matrix, long rows split into warp
        segments when that is faster) under the same protocol."""
        ct = run_steps(prep, K, 1, fn_name="csr")
        cms = sum(sum(v) for v in ct.values())
        cval = sum(2.0 * p["A"].nnz for p in prep) * K / (cms * 1e-3) / 1e9
        per = {}
        for p in prep:
            tc = statistics.median(ct[p["name"]])
            per[p["name"]] = {"group": p["csr_group"], "long_rows_split": p["csr_plan"] is not None,
                              "gflops": round(2.0 * p["A"].nnz / tc / 1e6, 1),
                              "gbs": round(csr_bytes(p, *VSIZE[key]) / tc / 1e6, 1),
                              "plain_gflops": round(2.0 * p["A"].nnz / p["csr_plain_ms"] / 1e6, 1),
                              "beta_over_csr": round(tc / statistics.median(beta_times[p["name"]]), 3)}
        return {"value": round(cval, 2), "unit": "GFLOP/s", "per_matrix": per,
                "speedup_beta_over_csr": round(beta_value / cval, 3)}

    def run_e2e(prep, K, stream, ws, dev, flops_step):
        """Pinned host x -> device, SpMV through the public call, y -> pinned host, every step."""
        hx = [torch.from_numpy(p["x"].cpu().numpy()).pin_memory() for p in prep]
        hy = [torch.empty(p["A"].n, dtype=p["y"].dtype).pin_memory() for p in prep]
        h2d = sum(t.numel() * t.element_size() for t in hx)
        d2h = sum(t.numel() * t.element_size() for t in hy)
        # three streams: host->device copies, the products, device->host copies;
        # events order each matrix's x copy before its product, its product before
        # its y copy, and keep the next step from overwriting a buffer still in use
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        nmat = len(prep)
        ev_x = [torch.cuda.Event() for _ in range(nmat)]    # x_j arrived
        ev_mv = [torch.cuda.Event() for _ in range(nmat)]   # product j done (x_j free, y_j ready)
        ev_y = [torch.cuda.Event() for _ in range(nmat)]    # y_j copied out (y_j free)
        for j in range(nmat):  # all "free" at the start
            ev_mv[j].record(stream)
            ev_y[j].record(stream)

        def e2e_step():
            for j, (p, a, b) in enumerate(zip(prep, hx, hy)):
                s_in.wait_event(ev_mv[j])
                with torch.cuda.stream(s_in):
                    p["x"].copy_(a, non_blocking=True)
                ev_x[j].record(s_in)
                stream.wait_event(ev_x[j])
                stream.wait_event(ev_y[j])
                p["M"].spmv(p["x"], p["y"], stream=stream)
                ev_mv[j].record(stream)
                s_out.wait_event(ev_mv[j])
                with torch.cuda.stream(s_out):
                    b.copy_(p["y"], non_blocking=True)
                ev_y[j].record(s_out)

        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            e2e_step()
        for j in range(nmat):  # the last copies out belong to the timed region
            stream.wait_event(ev_y[j])
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        return {"value": round(flops_step * K * ws / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "pinned host x in and y out every step on two copy streams, overlapping the products "
                            "(spc5_spmv on the compute stream); no L2 flush: x arrives through the copy (as it would "
                            "in a user's pipeline), the matrix arrays are cold because the other three matrices "
                            "(several GB) pass through L2 between two products of one matrix"}

    fp64_measured = spc5.fma_rate(torch.float64)  # live measured float64 FMA rate (GFLOP/s)
    peaks = spc5.device_peaks()
    hbm_nominal = peaks["hbm_gbs_nominal"]
    hbm_peak, hbm_src = measured_hbm_peak()
    prep64 = prepare(torch.float64)
    flops_step = sum(2.0 * p["A"].nnz for p in prep64)

    # ---- timed region (float64, selected formats)
    def timed_region():
        barrier(ws)
        torch.cuda.synchronize()
        with ClockSampler(local) as cs:
            w0 = time.perf_counter()
            t = run_steps(prep64, args.steps, args.warmup)
            torch.cuda.synchronize()
            w1 = time.perf_counter()
        torch.cuda.synchronize()
        barrier(ws)
        return t, cs.summary(), w0, w1

    times, clocks, wall0, wall1 = timed_region()
    # a run that saw a hardware or thermal slowdown is measured once more (every
    # rank together: the decision is the max over ranks)
    if max_over_ranks(1.0 if throttled(clocks) else 0.0, ws, dev) > 0:
        first = clocks
        times, clocks, wall0, wall1 = timed_region()
        clocks["remeasured_after"] = first["reasons"]
    step_ms = [sum(times[p["name"]][k] for p in prep64) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    value = flops_step * args.steps * ws / (total_ms * 1e-3) / 1e9
    # kernels of one product (as the library reports them) and the L2-flush copy before it
    launches_per_step = sum(p["M"].launch_count() + 1 for p in prep64)

    def roof(p, tlist, key):
        return roofline_entry(p, tlist, key, hbm_peak, hbm_src, hbm_nominal)

    per_matrix = [matrix_entry(p, times[p["name"]], "f64", hbm_peak) for p in prep64]
    dom = max(prep64, key=lambda p: statistics.median(times[p["name"]]))
    roofline = roof(dom, times[dom["name"]], "f64")
    # float64 on this GPU is also bounded by its float64 multiply-add rate
    dom_t = statistics.mean(times[dom["name"]])
    dom_gflops = 2.0 * dom["A"].nnz / dom_t / 1e6
    roofline["alu_fp64"] = {
        "achieved": round(dom_gflops, 1), "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
        "frac": round(dom_gflops / FP64_PEAK_GFLOPS, 4), "peak_measured": round(fp64_measured, 1),
        "frac_of_measured": round(dom_gflops / fp64_measured, 4),
        "why": "float64 multiply-adds run at 1/51 of the float32 rate on GB300: 2 flops per stored value need "
               "nnz/32 float64 warp-instructions, comparable to the HBM time of the value stream",
        "peak_source": "nominal float64 rate (2 FMA lanes/clk/SM x 152 SMs x 2.07 GHz x 2 = 1.25 TFLOP/s); "
                       "peak_measured by the library's multiply-add probe in this run"}

    # ---- CSR comparator, same protocol
    csr64 = csr_section(prep64, args.steps, "f64", value, times)

    # ---- end to end: pinned host x -> device, SpMV, y -> pinned host, every step
    e2e = run_e2e(prep64, args.steps, stream, ws, dev, flops_step)

    # ---- learned selector vs the paper-style polynomial on the bench matrices
    sel_res = run_selector_section(prep64, dev)

    # float64 products kept to report the error of the low-precision forms
    y64_ref = {p["name"]: p["M"].spmv(p["x"]).clone() for p in prep64}
    for p in prep64:
        p["M"].destroy()
        if p["csr_plan"] is not None:
            p["csr_plan"].destroy()
        del p["d"]
    torch.cuda.empty_cache()

    # ---- float32 and bfloat16 storage forms (x and y float32, float32 accumulation)
    low = {}
    for key, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        prep = prepare(dt)
        t = run_steps(prep, args.steps, 1)
        ms = sum(sum(v) for v in t.values())
        d = max(prep, key=lambda p: statistics.median(t[p["name"]]))
        sec = {"value": round(flops_step * args.steps / (ms * 1e-3) / 1e9, 1), "unit": "GFLOP/s",
               "hbm_gbs": round(sum(beta_bytes(p, *VSIZE[key]) for p in prep) * args.steps / (ms * 1e-3) / 1e9, 1),
               "per_matrix": [matrix_entry(p, t[p["name"]], key, hbm_peak, roofline=roof(p, t[p["name"]], key))
                              for p in prep],
               "roofline": roof(d, t[d["name"]], key)}
        sec["hbm_frac"] = round(sec["hbm_gbs"] / hbm_peak, 4)
        sec["csr"] = csr_section(prep, args.steps, key, sec["value"], t)
        sec["error_vs_float64"] = precision_errors(prep, y64_ref)
        for p in prep:
            p["M"].destroy()
            if p["csr_plan"] is not None:
                p["csr_plan"].destroy()
            del p["d"]
        torch.cuda.empty_cache()
        low[key] = sec

    # ---- precision form: float64 CG vs mixed-precision refinement, 7-point Poisson 96^3
    cg_res = run_cg_section(dev)
    cg_res["shifted"] = run_cg_section(dev, shifted=True)
    # ---- batched form: multi-RHS SpMM, float32; many uneven matrices in one launch
    spmm_res = run_spmm_section(mats, dev)
    batch_res = run_batch_section(dev)

    # ---- CPU baseline: the oracle as it stands, on the host cores, bounded sample
    cpu = run_cpu_baseline(mats, prep64) if rank == 0 else None

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "suite4 float64: " + ", ".join(p["name"] for p in prep64),
                   "formats": {p["name"]: f"beta({p['r']},{p['c']}) variant {p['variant']}" for p in prep64},
                   "selection": "exhaustive timing over the 12 shapes x kernel variants (the paper's best kernel)",
                   "l2": f"flushed before every SpMV ({L2_FLUSH_BYTES >> 20} MiB copy, outside the events)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "hbm_gbs": round(sum(beta_bytes(p, 8, 8) for p in prep64) * args.steps / (total_ms * 1e-3) / 1e9, 1),
        "hbm_peak": {"measured_gbs": hbm_peak, "measured_source": hbm_src, "nominal_gbs": round(hbm_nominal, 1),
                     "nominal_source": "2 x memory clock x bus width (driver attributes)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks, "wall_s_timed": round(wall1 - wall0, 3),
        "csr": csr64, "per_matrix": per_matrix, "f32": low["f32"], "bf16": low["bf16"], "cg": cg_res,
        "spmm_f32": spmm_res, "batch_f32": batch_res, "selector": sel_res,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
