"""Both builds stay free of compiler warnings: the oracle under strict C99
with every common warning, and the library's host code (each CUDA
translation unit, with the build's own flags) with -Wall -Wextra.  Warnings
are errors here.  CPU only: nothing runs, the objects are thrown away."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

from paper_2009_13569_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_compiles_without_warnings(tmp_path):
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-pedantic",
                           "-Wconversion", "-Werror", "-fPIC", "-c",
                           os.path.join(ROOT, "oracle", "oracle.c"), "-o",
                           str(tmp_path / "oracle.o")])


def test_cuda_host_code_compiles_without_warnings(tmp_path):
    def compile_one(src):
        obj = str(tmp_path / (src + ".o"))
        cmd = ([build._nvcc()] + build.ARCH + build.FLAGS +
               ["-Xcompiler", "-Wall,-Wextra,-Werror", "-c", os.path.join(build.CSRC, src),
                "-o", obj])
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        results = list(ex.map(compile_one, build._sources()))
    assert len(results) >= 8
    for src, rc, out in results:
        assert rc == 0 and "warning" not in out.lower(), "%s:\n%s" % (src, out[-2000:])
