"""Host-side pieces of bench.py on CPU: the clock summary parsed from
nvidia-smi's CSV (median SM clock, maximum, throttle reasons seen), the
traffic figure that is read from a committed ncu summary only while the
kernel sources still hash to the captured value, the algorithmic bytes of
one generation launch, and the reference arm's line (the oracle on the
host's cores)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def write_clock_rows(rows):
    path = f"/tmp/hsga_clocks_{os.getpid()}.csv"
    with open(path, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    return path


def row(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(smax), "900.00", "0x0000000000000000", hw, hwt, swt, cap]


def test_clock_summary_median_max_and_reasons(bench):
    write_clock_rows([row(2070, 2070), row(1965, 2070, cap="Active"), row(2070, 2070),
                      row(1800, 2070, hwt="Active"), ["garbage"]])
    s = bench.ClockSampler(0).summary()
    assert s["samples"] == 4                       # the malformed line is skipped
    assert s["sm_mhz"] == pytest.approx((1965 + 2070) / 2)
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(f"/tmp/hsga_clocks_{os.getpid()}.csv")


def test_clock_summary_without_samples_is_none(bench):
    write_clock_rows([])
    assert bench.ClockSampler(0).summary() is None
    assert bench.ClockSampler(0).summary() is None    # no file at all


def test_traffic_is_read_only_while_the_sources_match(bench, tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.kernel_source_hash(["kernel.cu"])
    prof = tmp_path / "profile.md"
    prof.write_text(f"notes\n\nsource_sha256: `{digest}`\ndram_bytes_per_launch: `123456`\n"
                    f"other_dram_bytes_per_generation: `789`\n")
    assert bench.profiled_traffic(profile=str(prof), sources=["kernel.cu"]) == 123456
    assert bench.profiled_traffic("other_dram_bytes_per_generation", str(prof),
                                  ["kernel.cu"]) == 789
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.profiled_traffic(profile=str(prof), sources=["kernel.cu"]) is None
    assert bench.profiled_traffic(profile=str(tmp_path / "missing.md"),
                                  sources=["kernel.cu"]) is None


def test_algorithmic_bytes_of_a_generation_launch(bench):
    agents = 512 * 1024 * 32
    assert bench.AGENTS == agents
    # 12-byte genome read and child written per agent, one 12-byte emigrant
    # gather per island
    assert bench.BYTES_PER_LAUNCH == agents * 24 + 512 * 1024 * 12 == 408_944_640


def test_reference_arm_prints_the_contract_line(bench):
    """`--impl reference` (the oracle on the host's cores) prints one JSON
    line with the same metric, unit and config as the GPU arm, its own
    cpu_baseline and an e2e object without host-device bytes; other ranks of
    a multi-process launch print nothing."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps",
           "1", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "agent replications/sec"
    assert d["unit"] == "agent replications/s" and d["higher_is_better"] is True
    assert d["config"] == bench.config_json(1)
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    other = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert other.returncode == 0 and not other.stdout.strip()
