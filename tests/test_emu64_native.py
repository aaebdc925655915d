"""The integer emulation of the binary64 squared distance used by the CUDA
distance kernel (csrc/emu64.cuh: the all-integer form, the mixed form and its
unrolled instances for d in {2, 3, 8, 16, 32}), compiled for the host,
against the host's own IEEE binary64 arithmetic on random tiles of many kinds
(unit cube, signed, integers with exact ties, spread binades, near-equal
values, zeros, signed zeros).  Exact equality of the bit patterns is
required."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("emu") / "emu64_check")
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-o", exe,
                           os.path.join(HERE, "native", "emu64_check.cpp")])
    return exe


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_emulation_bit_exact(checker, seed):
    out = subprocess.run([checker, str(seed), "20000"], capture_output=True, text=True)
    edges, bad, skipped = map(int, out.stdout.split())
    assert out.returncode == 0 and bad == 0, out.stderr
    assert edges > 3_000_000 and skipped < 20000 // 2
