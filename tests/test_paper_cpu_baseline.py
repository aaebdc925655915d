"""The paper-style multi-core CPU baseline (oracle/paper_cpu.c: OpenMP loops
over the distances and the de-duplication, a parallel merge sort, the
sequential column reduction; Sec. 3) gives exactly the oracle's bars, so the
benchmark compares the GPU path with a CPU program that computes the same
thing.  Runs on the CPU with several threads."""
import os

import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs


def _same(got, want):
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("make", [
    lambda: inputs.uniform(1, 3, seed=1),
    lambda: inputs.uniform(2, 3, seed=2),
    lambda: inputs.uniform(257, 3, seed=3),
    lambda: inputs.gaussian_mixture(613, 16, k=5, sigma=0.3, seed=4),
    lambda: inputs.lattice(12, 2),
    lambda: inputs.with_duplicates(300, 3, 37, seed=5),
    lambda: inputs.exponent_gaps(200, 5, seed=6),
    lambda: np.eye(40, dtype=np.float32),
])
def test_paper_cpu_baseline_equals_oracle(make):
    x = make()
    want, inf_v, nd = oracle.barcodes(x)
    got, inf_g, nd_g = oracle.barcodes_paper_cpu(x)
    _same(got, want)
    assert (inf_g, nd_g) == (inf_v, nd)


def test_paper_cpu_baseline_uses_threads_and_odd_thread_counts(monkeypatch):
    assert oracle.paper_cpu_threads() >= 1
    # an odd slice count exercises the unpaired run in the merge rounds
    x = inputs.noisy_circles(100, 3, 8, seed=7)
    want = oracle.barcodes(x)
    import subprocess
    import sys
    code = ("import oracle, numpy as np; from paper_2203_02527_gb300 import inputs; "
            "x = inputs.noisy_circles(100, 3, 8, seed=7); b, i, d = oracle.barcodes_paper_cpu(x); "
            "import sys; sys.stdout.buffer.write(b.tobytes())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                         env={**os.environ, "OMP_NUM_THREADS": "3"}, check=True).stdout
    assert out == want[0].tobytes()
