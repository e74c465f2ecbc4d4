"""The benchmark's reference arm on the host: `bench.py --impl reference` times the
CPU oracle running the whole benchmark estimate (Alg. 4.1 on the 5-level
hierarchy, same seed as the GPU arm) and prints one JSON line with the keys the
benchmark contract names; a rank other than 0 prints nothing and exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-9 * d["ms_per_step"]
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the GPU arm's workload and seed; N_l from Alg. 4.1's own variance estimates: at least the initial
    # 100 samples per level, and decreasing with the level as the variances of the corrections do
    import bench
    assert d["config"] == {"workload": bench.workload_desc(), "seed": bench.SEED}
    N = d["N_l"]
    assert len(N) == 5 and all(n >= 100 for n in N) and N[0] >= N[-1]
    assert d["rmse"] <= bench.TOL * 1.01 and 0.035 < d["estimate"] < 0.1


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
