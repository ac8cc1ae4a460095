"""The product path has no CPU fallback and does not reach the oracle: the
package's Python modules, CUDA sources and header import, include or load
nothing from oracle/ (the input generators only mention its conventions in
prose); a missing library raises; and without a GPU a sorter cannot be
created.  CPU only."""
import ast
import os

import pytest
import torch

from paper_2009_13569_gb300 import ipsgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2009_13569_gb300")


def _product_files(exts):
    for base in (PKG, os.path.join(ROOT, "include")):
        for d, _, files in os.walk(base):
            if "__pycache__" in d:
                continue
            for f in files:
                if f.endswith(exts):
                    yield os.path.join(d, f)


def test_package_python_never_imports_the_oracle():
    files = list(_product_files((".py",)))
    assert len(files) >= 4
    for path in files:
        with open(path) as f:
            tree = ast.parse(f.read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""] + [a.name for a in node.names]
            elif isinstance(node, ast.Constant) and isinstance(node.value, str):
                # no path to the oracle's library or sources in a string
                assert "liboracle" not in node.value and "oracle.c" not in node.value, path
                continue
            else:
                continue
            assert not any(n.split(".")[0] == "oracle" for n in names), path


def test_cuda_sources_and_header_do_not_reach_the_oracle():
    files = list(_product_files((".cu", ".cuh", ".h")))
    assert len(files) >= 10
    for path in files:
        with open(path) as f:
            text = f.read()
        for bad in ("oracle.h", "oracle.c", "liboracle", "oracle_"):
            assert bad not in text, (path, bad)


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(ipsgpu, "_lib", None)
    monkeypatch.setattr(ipsgpu, "LIB_PATH", str(tmp_path / "libipsgpu.so"))
    with pytest.raises(ipsgpu.IpsgpuError):
        ipsgpu.load()


@pytest.mark.skipif(torch.cuda.is_available(), reason="a GPU is present")
def test_without_a_gpu_a_sorter_cannot_be_created():
    from paper_2009_13569_gb300 import build
    build.build()
    with pytest.raises(ipsgpu.IpsgpuError) as e:
        ipsgpu.Sorter("u64")
    assert e.value.code == ipsgpu.E_CUDA
