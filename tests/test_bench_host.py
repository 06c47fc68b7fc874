"""Host-side pieces of bench.py that need no GPU: the algorithmic bytes per cell
the roofline divides by, the kernel each launch shape names, and the DRAM
traffic record's source check."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2305_05362_gb300 import workloads as wl  # noqa: E402


def test_bytes_per_cell():
    # disk: shared uniform mesh, residual on: read Q, read dv, write Q
    assert bench._bytes_per_cell(wl.disk(n_r=4, n_phi=512), 4) == 12
    assert bench._bytes_per_cell(wl.disk(n_r=4, n_phi=512), 8) == 24
    # batched rows: own meshes, no residual: Q in and out plus one 8-byte node
    w = wl.batched(n_rows=3, n_min=64, n_max=256)
    assert w.dv is None and not w.shared_mesh
    assert bench._bytes_per_cell(w, 4) == 16


@pytest.mark.parametrize("tuning,name", [
    ({"uniform_kernel_f32": 0, "rows_cells_per_thread_f32": 7}, "k_rows<float,3,7>"),
    ({"uniform_kernel_f32": 1, "seg_variant_f32": 0}, "k_useg<float,3,8,true,true>"),
    ({"uniform_kernel_f32": 1, "seg_variant_f32": 1}, "k_useg_pf<3,true,true>"),
    ({"uniform_kernel_f32": 1, "seg_variant_f32": 2}, "k_useg_ring<3,8,true,true>"),
    ({"uniform_kernel_f32": 2, "stream_cells_per_lane_f32": 8}, "k_stream<3,8>"),
])
def test_kernel_name(tuning, name):
    assert bench._kernel_name(tuning) == name


def test_traffic_record_matches_its_sources():
    """Every entry of the committed traffic record names existing sources; an
    entry is used only while their hash matches (otherwise traffic is null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    d = json.load(open(path))
    assert d
    for key, ent in d.items():
        kernel, workload = key.split(":")
        assert ent["dram_bytes_per_launch"] > 0
        h = hashlib.sha256()
        for rel in ent["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        got = bench._traffic(key)
        assert (got is not None) == (h.hexdigest() == ent["sha256"])
    assert bench._traffic("no_such_kernel:nowhere") is None


def test_traffic_is_about_the_algorithmic_bytes():
    """The recorded DRAM traffic of the disk kernels is within a few percent of
    the algorithmic bytes of one launch (12 B per cell; on the small disk the
    output stays in L2, so only the 8 B per cell read reach DRAM)."""
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, ent in d.items():
        if "disk_1024x4096" in key:
            cells = 1024 * 4096
            assert abs(ent["dram_bytes_per_launch"] / (8 * cells) - 1) < 0.02
        elif "disk_8192x16384" in key:
            cells = 8192 * 16384
            assert abs(ent["dram_bytes_per_launch"] / (12 * cells) - 1) < 0.02


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    one JSON line with the keys of the benchmark contract."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
