"""The radix sort's digit plan (csrc/ph0_common.cuh), compiled for the host
by nvcc: for key ranges of every width, the low digits cover the varying low
key bits exactly once, every digit fits its pass's radix, and a stable LSD
counting sort by the plan's digits orders random keys of the range exactly as
a comparison sort of (key, input index) does."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("plan") / "sort_plan_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2203_02527_gb300", "csrc"),
                           "-o", exe, os.path.join(HERE, "native", "sort_plan_check.cu")])
    return exe


@pytest.mark.parametrize("seed", [1, 2])
def test_plan_covers_and_sorts(checker, seed):
    out = subprocess.run([checker, str(seed)], capture_output=True, text=True)
    cases, bad = map(int, out.stdout.split())
    assert out.returncode == 0 and bad == 0, out.stderr
    assert cases > 300
