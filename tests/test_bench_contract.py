"""The bench's reference arm (the FP64 oracle on the host cores) runs without a
GPU, so its output line is checked here: one JSON line with every key of the
bench contract, the oracle described as the CPU baseline, and an end-to-end
figure without device copies.  Under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run({})
    assert len(lines) == 1
    r = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["value"] > 0 and r["ms_per_step"] > 0
    assert (r["n_gpus"], r["steps"], r["warmup"]) == (1, 1, 1)
    assert r["higher_is_better"] is True and r["scaling"] == "weak"
    # the default workload is the large image-patch one, with our arm's config
    sys.path.insert(0, ROOT)
    import bench
    assert r["config"]["workload"] == bench.WORKLOADS["patches"]
    assert (r["config"]["m"], r["config"]["K"], r["config"]["K1"], r["config"]["L"]) == (256, 1024, 512, 256)
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == r["value"]
    assert cb["extrapolated"] is True
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
