"""The reference arm of bench.py (the CPU oracle timed on the host cores) runs
without a GPU: one rank, and two gloo ranks under torchrun where rank 0 alone
prints the line and the other exits cleanly."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out: str):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def _check(line, n):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == n and line["unit"] == "GFLOP/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_one_rank():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--small", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 1)


def test_reference_arm_two_gloo_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--small", "--gpus",
           "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1  # rank 0 only
    _check(lines[0], 2)


def test_clock_samples_and_the_slowdown_rule():
    sys.path.insert(0, ROOT)
    import bench

    cs = bench.ClockSampler(0)
    # clocks.sm, clocks.max.sm, power, active-mask, hw, hw_thermal, sw_thermal, sw_power_cap
    cs.lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line"]
    s = cs.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and not bench.throttled(s)  # power cap: kept and noted
    cs.lines.append("1600, 2070, 1400.0, 0x8, Not Active, Active, Not Active, Not Active")
    s = cs.summary()
    assert "hw_thermal_slowdown" in s["reasons"] and bench.throttled(s)  # measured again
    assert not bench.throttled(bench.ClockSampler(0).summary())  # no samples at all


def test_bench_byte_counts_and_kernel_names():
    # the roofline's algorithmic bytes (values, column indices, masks, the two
    # interval arrays, x once, y) and the kernel names it reports per variant
    sys.path.insert(0, ROOT)
    import bench
    from paper_1801_01134_gb300 import inputs

    A = inputs.laplacian2d(10, 10)
    p = {"A": A, "r": 2, "c": 8, "nblocks": 37}
    I = (A.n + 1) // 2
    assert bench.beta_bytes(p, 8, 8) == 8 * A.nnz + (4 + 2) * 37 + 12 * (I + 1) + 8 * A.m + 8 * A.n
    assert bench.beta_bytes(p, 2, 4) == 2 * A.nnz + (4 + 2) * 37 + 12 * (I + 1) + 4 * A.m + 4 * A.n
    assert bench.csr_bytes(p, 4, 4) == 4 * A.nnz + 4 * A.nnz + 8 * (A.n + 1) + 4 * A.m + 4 * A.n
    names = {v: bench.spmv_kernel_names({"variant": v, "nseg": 0}) for v in (1, 5, 18, 22, 23, 25, 30, 32, 33)}
    assert names == {1: "k_spmv_rows", 5: "k_spmv_rows_u", 18: "k_spmv_rows_u", 22: "k_spmv_rows_g",
                     23: "k_spmv_rows_g", 25: "k_spmv_grp", 30: "k_spmv_rows_t", 32: "k_spmv_s", 33: "k_spmv_rows_g1"}
    assert bench.spmv_kernel_names({"variant": 30, "nseg": 3}) == "k_spmv_t_segs+k_spmv_fixup"
    assert bench.spmv_kernel_names({"variant": 1, "nseg": 3}) == "k_spmv_rows+k_spmv_segments+k_spmv_fixup"
