"""The benchmark's reference arm on the CPU: `bench.py --impl reference`
prints one JSON line with the contract's keys, the workload config of the GPU
arm, a cpu_baseline describing the run and an e2e entry with no host-device
traffic; warm-up below three steps is refused."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _bench(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=600, cwd=ROOT)


def test_reference_arm_line():
    res = _bench("--impl", "reference", "--steps", "2", "--warmup", "3")
    assert res.returncode == 0, res.stderr[-500:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 2
    assert line["higher_is_better"] is True and line["value"] > 0
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.config_json(bench.workload())
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_warmup_below_three_is_refused():
    res = _bench("--impl", "reference", "--steps", "2", "--warmup", "2")
    assert res.returncode != 0 and "warmup" in res.stderr
