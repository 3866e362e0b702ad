"""The benchmark's JSON contract, checked on the CPU through its reference arm
(the oracle timed on the host cores) on the small Laplacian workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
        "cpu_baseline", "e2e"}


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("method", ["kpm", "lanczos", "dgl"])
def test_reference_arm_line(method):
    line = run_bench("--impl", "reference", "--workload", "laplacian40", "--method", method,
                     "--steps", "1", "--warmup", "1")
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "laplacian40"


def test_algorithmic_bytes_formula():
    sys.path.insert(0, ROOT)
    import bench
    # Anderson 64^3, n_v = 64: CSR 1,835,008 x (4 + 4) + 4 (n + 1), three blocks of n x 64 floats
    assert bench.algorithmic_bytes_per_step(262144, 1835008, 64, "f32") == 217055236
    assert bench.fma_per_step(262144, 1835008, 64) == 1835008 * 64 + 4 * 262144 * 64


def test_roofline_names_the_variant_that_ran():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.step_kernel_name({"staged": 1, "chunk_bytes": 32}, "f32") == "step_kernel<float>"
    assert bench.step_kernel_name({"staged": 2}, "f64") == "step_staged_kernel<double>"
    assert bench.step_kernel_name({"staged": 3, "depth": 2}, "f32") == "step_tmag_kernel<float>"
    assert bench.step_kernel_name({"staged": 4, "chunk_bytes": 32}, "f32") == \
        "step_csrs_kernel<float>"
    assert bench.step_kernel_name(None, "f64") == "step_kernel<double>"


def test_cpu_baseline_reports_all_cores_and_one():
    """The oracle's rate on the host cores and on one thread, over bounded samples."""
    sys.path.insert(0, ROOT)
    import bench
    from synthetic import laplacian_2d
    cb = bench.cpu_baseline(laplacian_2d(40), -0.1, 8.1, 100, 20, 1, target_s=0.5)
    assert cb["kind"] == "oracle" and cb["unit"] == "moments/s" and cb["value"] > 0
    assert cb["cores"] >= 1 and "start vectors" in cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "1 thread" in st["sample"]


def test_panel_geometry_matches_the_library_rule():
    """Passes of at most w = min(panel or 256, 256) vectors, equal widths (the last may
    be narrower), rows padded to whole 16-byte chunks -- the rule of launch.panel."""
    import bench
    assert bench.panel_geometry(256, 0, "f32") == (1, 256, 256)
    assert bench.panel_geometry(20, 8, "f32") == (3, 7, 8)
    assert bench.panel_geometry(700, 0, "f32") == (3, 234, 236)
    assert bench.panel_geometry(700, 0, "f64") == (3, 234, 234)
    assert bench.panel_geometry(64, 16, "f64") == (4, 16, 16)
    assert bench.panel_geometry(5, 4096, "f32") == (1, 5, 8)
