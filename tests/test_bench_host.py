"""Host-side logic of bench.py (no GPU): the clock samples kept for the timed
region, and the shape of the reference arm's JSON line (the FP64 oracle timed
on host cores)."""
import datetime
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(t, mhz, power_cap="Not Active", hw="Not Active"):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, 0, {mhz}, 2070, 900.00, 0x0, {hw}, Not Active, Not Active, {power_cap}"


def test_clock_samples_kept_only_inside_the_timed_window():
    t = time.time()
    out = "\n".join([_row(t - 0.3, 1100), _row(t + 0.05, 2040), _row(t + 0.1, 2070, power_cap="Active"),
                     _row(t + 0.4, 1000, hw="Active"), "garbage line"])
    inside = bench.ClockSampler.parse(out, (t, t + 0.2))
    assert inside["samples"] == 2 and inside["samples_total"] == 4
    assert inside["sm_mhz"] == 2055.0 and inside["sm_max_mhz"] == 2070.0
    assert inside["reasons"] == ["sw_power_cap"]  # hw_slowdown fell outside the window
    everything = bench.ClockSampler.parse(out)
    assert everything["samples"] == 4 and "hw_slowdown" in everything["reasons"]
    empty = bench.ClockSampler.parse(out, (t + 1.0, t + 2.0))
    assert empty["samples"] == 0 and empty["sm_mhz"] is None
    assert bench.ClockSampler.parse("") is None
    # a timed region shorter than the sampling interval: the samples of the
    # same load right after it stand in, and the summary says so
    short = bench.ClockSampler.parse(out, (t + 0.01, t + 0.02), fallback=(t + 0.02, t + 0.2))
    assert short["samples"] == 2 and short["sm_mhz"] == 2055.0 and "right after" in short["note"]
    inside_first = bench.ClockSampler.parse(out, (t, t + 0.2), fallback=(t + 0.2, t + 1.0))
    assert inside_first["samples"] == 2 and "note" not in inside_first


@pytest.mark.parametrize("workload", [bench.DEFAULT_WORKLOAD, "autoencoder-bf16-b256"])
def test_reference_arm_prints_one_line_with_the_contract_keys(workload):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3", "--workload", workload], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "streams" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "streams", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == workload


@pytest.mark.parametrize("dtype,streams,expect", [("f32", 256, 1), ("bf16", 256, 1), ("bf16", 1024, 4),
                                                  ("f16", 2048, 8), ("bf16", 100, 1)])
def test_default_sub_batches(dtype, streams, expect):
    assert bench.default_sub_batches(dtype, streams) == expect


def test_model_memory_fields():
    class _Model:  # the two numbers cc_model_state_bytes reports
        state_bytes = (110592, 1081344)

    m = bench.model_memory(_Model(), 256, 9_000_000_000, 8_600_000_000)
    assert m == {"state_bytes_per_stream": 110592, "slot_bytes_per_stream": 1081344,
                 "arena_bytes": 1081344 * 256, "device_bytes_model": 400_000_000}
    assert bench.model_memory(_Model(), 1, None, None)["device_bytes_model"] is None
