"""The bench's JSON contract, checked on the CPU: the reference arm's line (the
oracle on the host cores), its silence on ranks other than 0 under torchrun,
the parser of the clock record sampled during the timed region, and the
whole-job aggregation of a single rank."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(*argv, **env_extra):
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], capture_output=True, text=True,
                          timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    out = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference"
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["metric"] == "Potts site-updates/s" and d["unit"] == "site-updates/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the same workload name as the default line of the GPU arm
    assert d["config"]["workload"] == "3d-1024-moore26-g1000000-plain-mcp-hybrid"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks():
    out = _run("--impl", "reference", "--steps", "1", "--warmup", "3", RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


class _FakeSmi:
    """Stands in for the nvidia-smi process: returns a canned CSV record."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_record_median_max_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1900, 2070, 1390.5, 0x8, Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 1390.5, 0x8, Not Active, Not Active, Not Active, Not Active",
        "not a record",
    ]
    c = bench.Clocks(0)
    c.proc = _FakeSmi("\n".join(rows))
    r = c.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070
    # "Not Active" must not count as active; each active reason is listed once
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_record_absent_without_a_sampler():
    assert bench.Clocks(0).stop() is None
    c = bench.Clocks(0)
    c.proc = _FakeSmi("")
    assert c.stop() is None


def test_whole_job_aggregate_of_one_rank():
    ms, v = bench.aggregate(2000.0, 10 ** 9, 1, "cpu")
    assert ms == 2000.0
    assert v == pytest.approx(5e8)
