"""The benchmark's reference arm (the FP64 oracle timed on the host cores) prints
one JSON line with the keys the measurement contract needs; CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_summary_keeps_every_extra_figure_compactly():
    """The line's last key repeats the extras' figures; the refined multi-group
    solve is set against its FP64-pipe bound (8 FP64 operations per element at the
    FP64 FMA rate measured in the same run) and the host link rates are kept."""
    sys.path.insert(0, ROOT)
    import bench
    ex = {"multigroup_refine": {"elements": 1000000, "refine2_fp64_residual": {
        "ms_per_call": 20.0, "launches": 1, "max_rel_err_per_group": [1e-16, 2e-16]}}}
    s = bench.summary(ex, {}, {}, None, 0, {"h2d": 211.0, "d2h": 193.0, "both": 341.0}, 8e8)
    assert s["multigroup_fp64_bound_ms"] == 10.0  # 1e6 x 8 / 8e8 s
    assert s["multigroup_of_fp64_bound"] == 0.5
    assert s["host_link_gbs"] == {"h2d": 211.0, "d2h": 193.0, "both": 341.0}
    assert s["multigroup_launches"]["refine2_fp64_residual"] == 1
    assert s["multigroup_max_err"] == 2e-16
    empty = bench.summary({}, {}, {}, None, 0)
    assert "multigroup_of_fp64_bound" not in empty and empty["host_link_gbs"] is None
