"""The benchmark's reference arm (the CPU oracle on the host cores) keeps the JSON-line contract;
under a multi-rank launch only rank 0 prints (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_json_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int),
                     ("steps", int), ("warmup", int), ("ms_per_step", float),
                     ("higher_is_better", bool), ("scaling", str), ("dtype", str),
                     ("data", str), ("config", dict), ("impl", str), ("cpu_baseline", dict),
                     ("e2e", dict)):
        assert isinstance(d[key], typ), key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["vs_baseline"] is None and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_sample_parsing():
    """The nvidia-smi sampling summary: median clock, max clock, throttle reasons seen Active,
    median power (the MDOF/W denominator); malformed lines are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    text = "\n".join([
        "2040, 2070, 900.5, Not Active, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1010.0, Active, Not Active, Not Active, Not Active, Active",
        "1990, 2070, [N/A], Active, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "",
    ])
    r = bench.parse_clock_samples(text)
    assert r["samples"] == 3 and r["sm_mhz"] == 2040 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]
    assert r["power_w"] == (900.5 + 1010.0) / 2
    assert bench.parse_clock_samples("") is None
