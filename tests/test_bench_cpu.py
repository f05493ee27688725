"""Host logic of bench.py: the clock summary, the roofline arithmetic, the size
of the reference arm's samples, and one short run of the reference arm (the
CPU oracle) checked against the JSON line's contract."""

import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# nvidia-smi rows in ClockSampler.FIELDS order: sm, max sm, power, then the
# hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap flags
ROWS = [
    "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
    "1965, 2070, 1399.0, Not Active, Not Active, Not Active, Active",
    "2070, 2070, 1210.2, Not Active, Not Active, Not Active, Not Active",
    "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",  # unparsable clock: skipped
    "garbage",
]


def test_parse_clocks_median_max_and_reasons():
    c = bench.parse_clocks(ROWS)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0  # median of 2070, 1965, 2070
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_parse_clocks_thermal_reason_and_empty():
    rows = ["1500, 2070, 1000, Not Active, Active, Not Active, Not Active"]
    assert bench.parse_clocks(rows)["reasons"] == ["hw_thermal_slowdown"]
    assert bench.parse_clocks([]) is None
    assert bench.parse_clocks(["x, y"]) is None


def test_roofline_mixed_bf16_is_the_method_flops_over_the_measured_bf16_rate():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1800.0}
    r = bench.roofline_for("mixed_bf16", 450.0, 3000.0, peaks, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1800.0)
    assert r["frac"] == pytest.approx(0.25)
    assert r["tensor_pipe_frac"] == pytest.approx(0.75)  # three bf16 products per algorithmic flop
    assert r["hbm"]["frac"] == pytest.approx(0.5)
    # without a sustained figure the burst rate stands in
    r = bench.roofline_for("mixed_bf16", 450.0, 3000.0, {"hbm_gbs": 6000.0, "bf16_tflops": 1500.0}, "x")
    assert r["peak"] == pytest.approx(1500.0)


def test_roofline_fp64_is_alu_bound():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    r = bench.roofline_for("fp64", 1.0, 100.0, peaks, "measured")
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(1.25) and r["frac"] == pytest.approx(0.8)


@pytest.mark.parametrize("cores", [1, 8, 16, 72])
def test_reference_samples_stay_bounded_for_any_step_count(cores):
    for steps in range(1, 200):
        per = bench.reference_points_per_step(cores, steps)
        assert per >= cores and per % cores == 0  # no process idles in the last round
        if steps <= 5:
            assert per == 5 * cores
        else:
            assert per * steps <= 25 * cores + cores * steps  # ~25 points per core in total


def test_reference_arm_prints_the_contract_line():
    cores = os.cpu_count() or 1
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--cpu-points", str(cores)], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["ms_per_step"] == pytest.approx(1e3 / line["value"])
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun rank 0 alone times the oracle and prints; the others exit 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=120,
                         cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_default_held_out_pairs_take_one_pair_on_each_side_of_the_mott_transition():
    u_mott = 2 ** 0.5
    pairs = bench.held_out_pairs(16)
    ins, met = bench.default_held_out_pairs(u_mott)
    assert ins[0] >= u_mott > met[0]
    # the first of each kind in the seeded held-out list, whatever its outcome
    assert ins == next(p for p in pairs if p[0] >= u_mott)
    assert met == next(p for p in pairs if p[0] < u_mott)
