"""The JSON contract of bench.py's reference arm, on CPU: the oracle timed on
the host cores prints one line with the metric, the value, its CPU-baseline
record and the e2e record (the small workload, and the paper-scale mixing
layer at a reduced size: the oracle decodes its blocks on demand, so the
full-size field needs no decoded copy either); a rank other than 0 prints
nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [json.loads(line) for line in p.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_line():
    lines = run(["--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = lines[0]
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "ms"
    assert d["higher_is_better"] is False and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOADS["small"]["name"]


def test_reference_arm_mixing_layer():
    lines = run(["--impl", "reference", "--workload", "paper", "--dims", "256", "256", "240",
                 "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and "unavailable" not in d
    assert d["config"]["dims"] == [256, 256, 240] and "256x256x240" in d["config"]["workload"]
    assert "on demand" in d["cpu_baseline"]["sample"]


def test_reference_arm_other_ranks_are_silent():
    lines = run(["--impl", "reference", "--workload", "small", "--steps", "1", "--warmup", "0"],
                {"RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def test_oracle_passes_line():
    """--oracle-passes times the oracle's raycaster with visible lists and its
    pass simulator; the counts it prints are the simulator's own."""
    lines = run(["--oracle-passes", "--workload", "small"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "oracle_passes" and d["cores"] >= 1
    assert d["render_with_lists_ms"] > 0 and d["simulate_ms"] >= 0
    assert d["passes"] >= 1 and d["blocks_decoded"] > 0 and d["entries"] > 0


def test_stage_rooflines_and_recorded_traffic():
    """The rooflines' arithmetic on made-up counters (bytes per unit times
    counts, over the stage time, against the peak), and every recorded DRAM
    traffic figure keyed by a kernel name the rooflines report, so that the
    line's `traffic` cannot silently become null after a rename."""
    import bench
    p = dict(n_processed=1000, n_entries_cap=4000, n_steps=20000, n_decoded=500, n_visible=300,
             n_entries=900)
    stage = {"traverse": 0.5, "decode": 0.25, "intersect": 0.125}
    rl = bench.stage_rooflines([(None, [p, p])], stage, 2, {"hbm_gbs": 1000.0})
    trav = 2 * (1000 * 80 + 4000 * 4 + 20000 * 8)
    dec = 2 * 500 * (8 * 2 + 256)
    isect = 2 * (300 * 500 + 900 * 24)
    for name, nbytes in (("traverse", trav), ("decode", dec), ("intersect", isect)):
        assert rl[name]["bytes"] == nbytes
        gbs = nbytes / 1e9 / (stage[name] / 1e3)
        assert abs(rl[name]["achieved"] - round(gbs, 1)) < 1e-9
        assert abs(rl[name]["frac"] - round(gbs / 1000.0, 4)) < 1e-12
    kernels = {v["kernel"] for v in rl.values()}
    for (kernel, dims, rate), (nbytes, source) in bench.MEASURED_TRAFFIC.items():
        assert kernel in kernels, kernel
        assert tuple(dims) == bench.WORKLOADS["paper"]["dims"] and rate == bench.WORKLOADS["paper"]["rate"]
        assert nbytes > 0 and "ncu" in source
