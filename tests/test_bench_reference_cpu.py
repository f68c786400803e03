"""bench.py's reference arm (the oracle timed on the host cores) on CPU: the JSON line it prints and
the rank rule (only rank 0 of a multi-rank launch runs and prints)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    if extra_env:
        env.update(extra_env)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "200", "--steps", "2",
                           "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "pair-interactions/s" and line["unit"] == "pair-interactions/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert "N_m=200" in line["config"]["workload"]
    # the GPU arm's window: the same warm-up steps untimed, then exactly the timed steps, and the
    # same workload string
    assert line["steps"] == 2 and line["warmup"] == 3
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    ns = argparse.Namespace(n=200, n_field=0, precision="fp64", seed=1002)
    assert line["config"]["workload"] == bench.workload_name(ns)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert cb["unit"] == "pair-interactions/s" and cb["sample"]
    pk = cb["parallel_kick"]
    assert pk["pairs_per_s"] > 0 and pk["threads"] >= 1 and pk["ms_per_kick"] > 0
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
