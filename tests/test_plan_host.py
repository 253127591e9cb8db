"""Host logic of the tensor-core work split, checked on the CPU: tests/plan_check.cu
includes the library's host source, is compiled with nvcc against the built library
and run without a GPU (the planner does no device work). It checks that every pair of
the evaluated triangle is in exactly one work unit, that the merge reads only row-side
list slots written exactly once, the band units, the phases of a host-buffer call and
the default work-unit length."""
import os
import shutil
import subprocess

import pytest

import paper_2603_02059_gb300 as tk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    path = shutil.which("nvcc")
    if path is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        path = "/usr/local/cuda/bin/nvcc"
    return path


def test_work_plan_host_checks(tmp_path):
    tk.lib()  # the built library (raises with the build command if it is missing)
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    libdir = os.path.dirname(tk.LIB_PATH)
    exe = str(tmp_path / "plan_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-o", exe,
           os.path.join(ROOT, "tests", "plan_check.cu"), "-L", libdir, "-ltraknn",
           "-Xlinker", "-rpath", "-Xlinker", libdir]
    build = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout[-3000:] + run.stderr[-2000:]
    assert "plan check ok" in run.stdout
