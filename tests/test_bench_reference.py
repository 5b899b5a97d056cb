"""bench.py's reference arm (the FP64 CPU oracle timed on the host) keeps the
JSON contract of the benchmark line, on a small grid so that it runs in seconds;
under torchrun only rank 0 runs it."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "63",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=300)
    return out


def test_reference_line_keeps_the_contract():
    out = run_bench()
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["higher_is_better"] is True
    for key in ("metric", "value", "n_gpus", "steps", "ms_per_step", "scaling", "vs_baseline", "dtype", "data",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    # at a grid no larger than the sample size nothing is extrapolated: the steps
    # are complete solves and the rate is steps / wall
    assert line["value"] > 0 and abs(line["ms_per_step"] - 1e3 / line["value"]) <= 1e-9 * line["ms_per_step"]
    # the claimed timed work fits inside the run
    assert line["steps"] * line["ms_per_step"] <= 1e3 * line["wall_s"]
    cb = line["cpu_baseline"]
    assert cb["measured"]["solves"] == line["steps"] and cb["measured"]["n"] == 63
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "grf_63"


def test_reference_arm_runs_on_rank_zero_only():
    out = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_traffic_record_matches_the_committed_profiles():
    """The DRAM traffic that bench.py reports next to the roofline comes from the
    committed ncu summary only while the kernel's source is the one profiled
    (its hash is recorded beside the number); the committed summary is current."""
    sys.path.insert(0, ROOT)
    import bench
    for kernel in ("residual_kernel", "down_kernel", "up_kernel"):
        t = bench.traffic_record(kernel, "grf_4095")
        assert t is not None and t > 1e8, f"{kernel}: profiles/dram_traffic.txt is stale, re-profile"
    assert bench.traffic_record("up_kernel", "channelised_4095") is None
    assert bench.traffic_record("no_such_kernel", "grf_4095") is None


def test_algorithmic_bytes_per_unknown():
    """The per-unknown byte counts behind the roofline (8 channels, BF16 state,
    FP64 u, f and stencil): residual 60 (u, f, five stencil planes in; FP32 r
    out), finest down 40 (FP32 r, s in; x_down, coarse x out), finest up 56
    (x_down, s, the coarse x_fin's high and low parts, u in; u out), coarser
    down 52 and up 72 per level unknown (the up sweep's x_fin in and out as high
    and low parts); the coarse tail sums its levels."""
    sys.path.insert(0, ROOT)
    import bench
    n = 4095
    N = n * n
    assert bench.algorithmic_bytes("residual", n, 8) == 60 * N
    assert bench.algorithmic_bytes("down0", n, 8) == 40 * N
    assert bench.algorithmic_bytes("up0", n, 8) == 56 * N
    assert bench.algorithmic_bytes("down1", n, 8) == 52 * 2047 * 2047
    assert bench.algorithmic_bytes("up2", n, 8) == 72 * 1023 * 1023
    levels = [255, 127, 63, 31, 15, 7, 3]
    assert bench.algorithmic_bytes("tail", n, 8) == sum((52 + 72) * m * m for m in levels)


def test_omega_argument_and_record():
    """--omega takes one Jacobi weight or three (finest, in between, coarsest); the
    bench line records them for the analytic networks only."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_omega("0.8") == 0.8
    assert bench.parse_omega("0.8,1.5,1.0") == (0.8, 1.5, 1.0)
    with pytest.raises(SystemExit):
        bench.parse_omega("0.8,1.5")
    assert bench.omega_record((0.8, 1.5, 1.0), "gmg_v10") == {"finest": 0.8, "in_between": 1.5, "coarsest": 1.0}
    assert bench.omega_record(0.8, "gmg") == 0.8
    assert bench.omega_record((0.8, 1.5, 1.0), "trained") is None
