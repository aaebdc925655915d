"""The large-cloud edge records: above 65535 points an edge's record holds
its lexicographic index e = u(2n-u-1)/2 + v-u-1, and the kernels recover
(u, v) from e (csrc/ph0_common.cuh, record_uv).  Compiled for the host by
nvcc and checked against the index formula on every edge of small clouds and
on every row's first and last edges up to n = 92681."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_edge_index_decoding(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    exe = str(tmp_path / "edge_index_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2203_02527_gb300", "csrc"),
                           "-o", exe, os.path.join(HERE, "native", "edge_index_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert checked > 10_000_000
