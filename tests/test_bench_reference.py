"""bench.py's reference arm (the FP64 oracle on the host cores, one process
per allowed core) prints one contract line on rank 0 and nothing on the other
ranks; the all-core timing sums the processes' rates (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "dipole64",
                           "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "Mcell-updates/s" and d["unit"] == "Mcell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["config"]["workload"].startswith("passive fcc opal 2x2x2")
    cb = d["cpu_baseline"]
    # one oracle process per allowed core (fewer only when host memory is short)
    assert cb["kind"] == "oracle" and 1 <= cb["cores"] <= len(os.sched_getaffinity(0))
    assert cb["value"] == d["value"] and f"{cb['cores']} processes" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_all_core_oracle_timing_sums_independent_realizations():
    import bench
    from paper_0802_3775_gb300 import inputs
    specs = [inputs.opal_dipole_f64(steps=4) for _ in range(2)]
    rate, per = bench.time_oracle_all_cores(specs, steps=3, warmup=1)
    assert [n for n, _ in per] == [3, 3]
    assert abs(rate - sum(s.cells * n / t for s, (n, t) in zip(specs, per)) / 1e6) < 1e-9 * rate
