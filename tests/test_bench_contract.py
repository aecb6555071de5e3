"""CPU checks of the benchmark's reference arm (the FP64 oracle timed on the
host): one JSON line with the contract's keys, and silence on ranks other
than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
        "--cpu-detscans", "4", "--ref-detscans-per-step", "1"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(ARGS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    p = _run({})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["steps"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["unit"] == d["e2e"]["unit"] == "samples/s"
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_cg_pass_bytes_follow_the_launched_iterations():
    """The algorithmic bytes of the CG passes: iteration i of a flagged
    detscan runs in launch i while i < launched, the rest in the cooperative
    tail; the correction passes cover every detscan that ran the CG."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    lens = np.array([100.0, 200.0, 300.0, 400.0])
    iters = np.array([1, 3, 10, 0])
    flagged = np.array([True, True, True, False])
    kb = bench.kernel_bytes(1000, 10, 5, 0, lens, iters, flagged, launched=8)
    # launched iterations: detscan 0 once, 1 three times, 2 eight times
    act = 100 * 1 + 200 * 3 + 300 * 8
    assert kb["k_nc_filter"] == 8.0 * act
    assert kb["k_nc_scatter"] == 4.0 * act
    assert kb["k_nc_gather"] == 4.125 * act
    assert kb["k_nc_tail"] == 16.125 * 300 * 2
    assert kb["k_nc_filter_final"] == 8.0 * (100 + 200 + 300)
    kb3 = bench.kernel_bytes(1000, 10, 5, 0, lens, iters, flagged, launched=3)
    assert kb3["k_nc_filter"] == 8.0 * (100 + 200 * 3 + 300 * 3)
    assert kb3["k_nc_tail"] == 16.125 * 300 * 7
