"""The reference arm of bench.py (the CPU oracle on the host cores) prints
one JSON line with the keys the measurement contract names, and a non-zero
rank of a multi-process launch exits without work or output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0", "--ref-seconds", "0.2", "--D", "4",
                           *args], capture_output=True, text=True, env=env, timeout=600,
                          cwd=ROOT)


def test_reference_arm_prints_the_contract_line():
    out = _run()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "NTU bond updates/s" and d["unit"] == "bond updates/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert isinstance(d["dtype"], str)
    assert d["config"]["workload"].startswith("batched NTU bond updates, D=4")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    out = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_environment_roofline_names_its_peak():
    sys.path.insert(0, ROOT)
    import bench
    m = bench.env_roof("bf16x3", 950e12, {"bf16_tflops": 1900.0})
    assert m["frac"] == 0.5 and m["issued_frac"] == 1.5 and "measured" in m["peak_source"]
    f = bench.env_roof("bf16x3", 950e12, {})
    assert f["peak"] == 1900.0 and "fallback" in f["peak_source"]
    a = bench.env_roof("fp64", 1.1e12, {"fp64_tflops": 1.1})
    assert a["bound"] == "alu" and abs(a["frac"] - 1.0) < 1e-12 and "measured" in a["peak_source"]


def test_als_roofline_counts_the_contraction_against_measured_peaks():
    """The ALS roofline credits the reduced-problem contractions of every
    sweep, 2 (K^4 D + K^3 D^2) complex multiply-adds, and divides by the
    measured ceiling of the pipe they run on (FP32 lanes for the double-FP32
    build of the mixed contexts, FP64 otherwise)."""
    sys.path.insert(0, ROOT)
    import bench
    K, D = 16, 8
    assert bench.als_flops(D, 2, 10) == 10 * 2 * 8.0 * (K ** 4 * D + K ** 3 * D * D)
    pk, src = bench.als_peak("bf16x3", {"fp32_tflops": 70.0, "fp64_tflops": 1.1})
    assert pk == 70.0e12 and "measured fp32" in src
    pk, src = bench.als_peak("fp64", {"fp32_tflops": 70.0, "fp64_tflops": 1.1})
    assert pk == 1.1e12 and "measured fp64" in src


def test_oracle_leg_returns_the_accuracy_sample():
    """The CPU-baseline leg times the oracle in a child process and hands
    back its results for the sampled items; comparing them with themselves
    gives zero error, and a perturbed metric shows up in g_rel_frob_max."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rate, n, sec, th, kept = bench._oracle_rate(3, 2, 2, 0.05, 5, max_items=3, threads=1,
                                                keep=[0, 2], batch=3)
    assert rate > 0 and n >= 2 and th == 1
    assert set(kept) == {"g0", "A0", "B0", "d0", "x0", "g2", "A2", "B2", "d2", "x2"}
    gpu = {"g": np.stack([kept["g0"], kept["g2"] * (1 + 1e-6)]),
           "A": np.stack([kept["A0"], kept["A2"]]), "B": np.stack([kept["B0"], kept["B2"]]),
           "info": np.array([[0, kept["d0"][0], 0, 0], [0, kept["d2"][0], 0, 0]]),
           "sx": np.array([kept["x0"][0], kept["x2"][0]])}
    acc = bench.accuracy_vs_oracle(gpu, kept, [0, 2])
    assert abs(acc["g_rel_frob_max"] - 1e-6) < 1e-12
    assert acc["delta_rel_max"] == 0 and acc["pair_rel_max"] == 0 and acc["sx_abs_max"] == 0
