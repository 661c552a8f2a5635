"""Host-side parts of bench.py that need no GPU: the reference arm's JSON
line (the oracle timed on the host cores), the all-cores CPU leg (one
oracle copy per core), the unit conversion of the metric, the per-launch
byte counts of the integrator and the guard that reports the adjoint's DRAM
traffic only while its sources are the captured ones."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_ns_per_day():
    # one 10 fs step per second: 10 fs x 86,400 s/day = 864,000 fs = 0.864 ns
    assert bench.ns_per_day(10.0, 1.0) == pytest.approx(0.864, rel=1e-12)
    assert bench.ns_per_day(1.0, 1000.0) == pytest.approx(86.4, rel=1e-12)


def test_integrator_bytes_per_outer_step():
    # per atom: an inner launch 57 B read + 24 B written, the outer-kick launch
    # 12 B more read, the closing launch 40 + 12
    assert bench.integ_bytes_per_outer_step(5, False) == 93 + 4 * 81
    assert bench.integ_bytes_per_outer_step(5, True) == 93 + 4 * 81 + 52
    assert bench.integ_bytes_per_outer_step(1, False) == 93


def test_serving_roofline_counts_the_integrator_bytes():
    # one tick = one call of one outer step: n_inner launches and the
    # closing one; 1e6 atom-outer-steps in 1 ms of integrator time
    from paper_2602_14975_gb300 import synth as S
    cs = S.cons_spec(3, 128, 2)
    prof = {"integrate": (6, 1.0), "gemm_tc": (14, 2.0)}
    out = bench.serving_roofline(prof, 1e6, 5, cs)
    assert out["integrate"]["gbs"] == pytest.approx((93 + 4 * 81 + 52) * 1e6 / 1e-3 / 1e9)
    flop = 2.0 * 128 * 128 * (2 * 3 * 4 + 2) * 1e6
    assert out["gemm_tc"]["tflops"] == pytest.approx(flop / 2e-3 / 1e12)
    assert out["shares"] == {"gemm_tc": pytest.approx(2 / 3, abs=1e-4), "integrate": pytest.approx(1 / 3, abs=1e-4)}


def test_adjoint_traffic_only_for_the_captured_sources():
    rec = bench.NCU_TRAFFIC["mp_bwd"]
    if bench.sources_sha256(rec["sources"]) == rec["sha256"]:
        assert bench.ncu_traffic("mp_bwd") == pytest.approx(rec["bytes_per_launch"])
    else:
        assert bench.ncu_traffic("mp_bwd") is None
    stale = dict(rec, sha256="0" * 64)
    bench.NCU_TRAFFIC["stale_probe"] = stale
    try:
        assert bench.ncu_traffic("stale_probe") is None
    finally:
        del bench.NCU_TRAFFIC["stale_probe"]
    assert bench.ncu_traffic("no_such_kernel") is None


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "ns/day" and line["value"] > 0
    assert line["config"]["workload"] == "solvated_chain_23558"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_all_cores_leg_runs_one_oracle_copy_per_usable_cpu():
    """The all-cores CPU figure: the unmodified oracle in one spawned process
    per CPU this process may use, on the same periodic sample; its rate is
    the sum of the copies' rates (each scaled to the full system)."""
    from paper_2602_14975_gb300 import synth as S
    W = S.WORKLOADS["solvated_chain_23558"]
    sy = S.WORKLOADS["water_12288"]["system"]()
    rate, p, wall, desc = bench.oracle_all_cores(sy, W, 0.3)
    assert p == bench.usable_cpus() >= 1
    assert rate > 0.0 and wall > 0.0
    assert f"{p} concurrent copies" in desc
