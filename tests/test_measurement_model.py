"""The byte model behind the benchmark's rooflines, against the I/O volume
the paper prints for the in-place samplesort (tests/golden): every level
reads and writes each element once in classification and once in the block
permutation, the base case once more (no write allocates)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "io_volume_ips4o.txt")


def _table():
    facts = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                facts[k] = int(v)
    return facts


def test_level_bytes_match_the_papers_io_table():
    sys.path.insert(0, ROOT)
    import bench
    t = _table()
    D, n = t["element_bytes"], 1 << 20
    # per-kernel algorithmic bytes as the library reports them: 2 D per
    # element for classification and for the permutation, per level
    levels = 2
    stats = {"classify": (levels, 1.0, levels * 2.0 * D * n),
             "permute": (levels, 1.0, levels * 2.0 * D * n),
             "sample_tree": (levels, 0.1, 0.0)}
    lv = bench.level_roofline(stats, 6704.5, D, n)
    per_level = t["classification_per_level"] + t["redistribution_per_level"]
    assert lv["bytes"] == pytest.approx(levels * per_level * n)
    assert lv["levels"] == pytest.approx(levels)
    # the base case: one read and one write of every element
    assert t["base_case_once"] == 2 * D


def test_traffic_model_is_per_element():
    sys.path.insert(0, ROOT)
    import bench
    # the scaled traffic of a kernel is its measured bytes per element times
    # the elements of a launch (None when the source changed since capture)
    t = bench.NCU_TRAFFIC["classify"]
    assert 14.0 < t["bytes_per_elem"] <= 16.0  # at most the 2 x 8 B of the model
    got = bench._traffic("classify", 1 << 20)
    assert got is None or got == pytest.approx(t["bytes_per_elem"] * (1 << 20))


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback(monkeypatch, tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    import json
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6704.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peak_hbm() == (6704.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    assert bench._peak_hbm() == (6800.0, "fallback")  # the recipe's fallback figure
    (tmp_path / "MEASURED_PEAKS.json").write_text("{}")
    assert bench._peak_hbm() == (6800.0, "fallback")


def test_traffic_is_null_once_the_kernel_source_changes(monkeypatch, tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cuh"
    src.write_text("kernel v1\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k": {"bytes_per_elem": 15.0, "source": "k.cuh",
                                                     "sha256": sha}})
    assert bench._traffic("k", 1000) == pytest.approx(15000.0)
    src.write_text("kernel v2\n")
    assert bench._traffic("k", 1000) is None
    assert bench._traffic("other", 1000) is None
