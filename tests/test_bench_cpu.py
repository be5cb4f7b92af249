"""The benchmark's reference arm (the oracle timed on the host) and its JSON
line, run on the CPU: the keys the line must carry, the bounded sample it
states, and that under a multi-rank launch only rank 0 runs and prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*argv, env_extra=None, timeout=300):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=timeout)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    return lines


def _check_line(line, steps, warmup, unit):
    sys.path.insert(0, ROOT)
    import bench

    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["unit"] == unit
    assert line["value"] > 0
    assert line["n_gpus"] == 1
    assert (line["steps"], line["warmup"]) == (steps, warmup)
    assert line["higher_is_better"] is True
    assert line["vs_baseline"] is None
    assert line["data"] == "synthetic"
    assert line["config"]["workload"]
    # the sample is bounded: the line says what one step was
    assert line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["sample"]
    assert cb["value"] == line["value"] and cb["unit"] == unit
    assert cb["host"]["model"] and cb["host"]["nproc"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == unit
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_single_graph():
    lines = _bench("--impl", "reference", "--workload", "gnm14", "--steps", "3", "--warmup", "3")
    assert len(lines) == 1
    line = json.loads(lines[0])
    _check_line(line, 3, 3, "GTEPS")
    # the same config object and e2e unit as the GPU arm prints, so the two
    # lines can be compared key by key
    import bench

    w = bench.WORKLOADS["gnm14"]
    xadj, adj = bench.make_graph(w)
    assert line["config"] == bench.bench_config(w, len(xadj) - 1, len(adj), 1)
    assert line["e2e"]["unit"] == bench.E2E_UNIT


def test_reference_arm_batch():
    lines = _bench("--impl", "reference", "--workload", "batch4096", "--steps", "1", "--warmup",
                   "0")
    assert len(lines) == 1
    line = json.loads(lines[0])
    _check_line(line, 1, 0, "graphs/s")
    assert "16 graphs" in line["cpu_baseline"]["sample"]


def test_reference_arm_serve_is_marked_unavailable():
    lines = _bench("--impl", "reference", "--workload", "serve", "--steps", "1", "--warmup", "0")
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unavailable"]


@pytest.mark.parametrize("workload", ["gnm14", "batch4096"])
def test_reference_arm_other_ranks_do_no_work(workload):
    lines = _bench("--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "0",
                   env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []


def test_profile_summary_fields():
    """The committed lane-kernel summary carries what the bench reads from
    it, and the traffic it reports is either that figure or null."""
    sys.path.insert(0, ROOT)
    import bench

    path = os.path.join(ROOT, "profiles", "rate_lane_rgg24.txt")
    fields = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                fields[k.strip()] = v.strip()
    assert len(fields["source_hash"]) == 16
    assert float(fields["dram_bytes_per_launch"]) > 0
    t = bench.ncu_traffic("rate_lane", "rgg24")
    if fields["source_hash"] == bench.kernel_source_hash("rate"):
        assert t == float(fields["dram_bytes_per_launch"])
    else:
        assert t is None


def test_host_cpu_from_arm_cpuinfo(monkeypatch, tmp_path):
    # Arm kernels list implementer and part numbers instead of a model name
    fake = tmp_path / "cpuinfo"
    fake.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\n"
                    "CPU part\t: 0xd4f\n\nprocessor\t: 1\nCPU part\t: 0xd4f\n")
    real_open = open

    def fake_open(path, *a, **k):
        return real_open(fake if path == "/proc/cpuinfo" else path, *a, **k)

    monkeypatch.setattr("builtins.open", fake_open)
    sys.path.insert(0, ROOT)
    import bench

    h = bench.host_cpu()
    assert "implementer 0x41" in h["model"] and "part 0xd4f" in h["model"]
    assert h["nproc"] >= 1
