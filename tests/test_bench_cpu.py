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


def test_roofline_attribution_helpers():
    # which kernel a workload's roofline line is about, the share of the updates
    # it makes and its algorithmic bytes per update
    sys.path.insert(0, ROOT)
    import bench

    W = bench.WORKLOADS
    assert bench.kernel_name(W["pa-ising2d-L64"], {"sweep_bits": (1, 1.0)}) == "sweep_bits"
    assert bench.kernel_name(W["pa-ising2d-L64"], {"sweep_resident": (1, 1.0)}) == "sweep_resident"
    assert bench.kernel_name(W["ising2d-L4096"], {"bitpack_strips": (1, 1.0), "bitpack_convert": (2, 0.1)}) == \
        "bitpack_strips"
    assert bench.kernel_name(W["ising2d-L4096"], {"sweep_strips": (1, 1.0)}) == "sweep_strips"
    assert bench.kernel_name(W["ising2d-L4096-sw"], {"swendsen_wang": (3, 1.0)}) == "swendsen_wang"
    assert bench.kernel_name(W["ising2d-L4096-dcb"], {"sweep_dcb_resident": (1, 1.0)}) == "sweep_dcb_resident"
    assert bench.kernel_name(W["ising2d-L4096-dcb"], {"sweep_dcb_bits": (2, 1.0)}) == "sweep_dcb_bits"
    assert bench.kernel_name(W["ising2d-L4096-dcb"], {"sweep_dcb": (2, 1.0)}) == "sweep_dcb"
    # every lattice of the mixed batch is one the bit-sliced kernel sweeps
    assert bench.dominant_share(W["pa-mixed-2d"], "sweep_bits") == 1.0
    mixed = dict(W["pa-mixed-2d"], lattices=[(2, 24, 0, 1, 1000), (2, 64, 0, 1, 1000)])
    share = bench.dominant_share(mixed, "sweep_bits")
    assert abs(share - 64 ** 2 / (24 ** 2 + 64 ** 2)) < 1e-12
    assert abs(bench.dominant_share(mixed, "sweep_resident") + share - 1.0) < 1e-12
    # PA: a copy read and written once per theta sweeps, plus E, M and its parent
    b = bench.alg_bytes_per_update(W["pa-ising2d-L64"], "sweep_bits")
    assert abs(b - (2 * 4096 + 12) / (4096 * 10)) < 1e-12
    assert bench.alg_bytes_per_update(W["ising2d-L4096-sw"], "swendsen_wang") == 7.0
    # double checkerboard, 64 x 64 tiles, k = 10: the bit-sliced tile reads a
    # one-site halo, the byte-plane window an 8-site one
    assert abs(bench.alg_bytes_per_update(W["ising2d-L4096-dcb"], "sweep_dcb_bits") - (2 + 4 / 64) / 10) < 1e-12
    assert abs(bench.alg_bytes_per_update(W["ising2d-L4096-dcb"], "sweep_dcb_resident") -
               (2 / 1000 + 0.75 / 640)) < 1e-12
    assert abs(bench.alg_bytes_per_update(W["ising2d-L4096-dcb"], "sweep_dcb") - (80 ** 2 + 64 ** 2) / 64 ** 2 / 10) \
        < 1e-12


def test_gpu_record_line_from_a_run_result():
    # the JSON line of a GPU workload from a (synthetic) run result: contract keys,
    # value = site updates / time, and the roofline of the dominant kernel
    sys.path.insert(0, ROOT)
    import bench

    w = dict(bench.WORKLOADS["ising2d-L4096-dcb"])
    upd = 4096 ** 2 * 1000
    res = dict(ms=12.0 * 2, steps=2, warmup=3, upd_all=2.0 * upd, upd_local=2.0 * upd, upd_prof=2.0 * upd,
               ms_profiled=24.5, prof={"sweep_dcb_bits": (400, 24.0)}, launches=400,
               clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, sm_count=152)
    line = bench.gpu_record(w, "ising2d-L4096-dcb", res, 1)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks"):
        assert k in line, k
    assert abs(line["value"] - upd / (12.0 * 1e6)) < 1e-9 and line["ms_per_step"] == 12.0
    roof = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["kernel"] == "sweep_dcb_bits" and roof["bound"] == "alu"
    # 20 algorithmic integer ops per update over the kernel's own 24 ms
    assert abs(roof["achieved"] - 20.0 * 2 * upd / 24e-3 / 1e9) < 1e-6
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    assert line["config"]["workload"] == "ising2d-L4096-dcb" and line["gpu_launches"] == 400
