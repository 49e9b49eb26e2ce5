"""The benchmark's reference arm (the FP64 oracle on the host's cores) runs
without a GPU and prints the JSON line of the benchmark contract: the same
metric, unit and direction as the GPU arm, its CPU baseline, and an e2e
entry with no host-device copies (CPU, about 20 s)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("fwd+bwd ms/view") and d["unit"] == "Gpoints/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["n_gpus"] == 1
    assert (d["steps"], d["warmup"]) == (1, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["data"] == "synthetic" and d["vs_baseline"] is None
    assert d["config"]["n_samples"] == 4194304 and d["config"]["image"] == [1280, 832]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_loads_only_the_oracle():
    # the reference arm sizes its table with the oracle's layout rule and
    # maps no library of the GPU path
    code = ("import sys, types, bench; a = types.SimpleNamespace(steps=1, warmup=0, gpus=1); "
            "bench.run_reference(a, 0); maps = open('/proc/self/maps').read(); "
            "sys.exit(3 if 'libinpc' in maps else (0 if 'liboracle' in maps else 4))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
