"""The benchmark's reference arm (the CPU oracle on a bounded sample) prints
one JSON line with the keys the result contract names, for a PA workload, a
single-lattice workload and parallel tempering."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["ising2d-L4096-sw", "pa-ising2d-L64-nearest", "pt-ea3d-L8"])
def test_reference_arm_json_line(workload):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == workload
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_all_cores_oracle_timing_runs_one_sample_per_core():
    sys.path.insert(0, ROOT)
    import bench

    w = dict(kind="sweeps", dim=2, L=64, sweeps=2, beta=0.44, layout=0)
    v, cores, seconds = bench.cpu_oracle_all_cores(w)
    assert cores >= 1 and seconds > 0 and v > 0
