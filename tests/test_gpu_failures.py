"""Failure detection without a GPU fault: a bounded device wait that runs
out, and an allocation that fails, are reported as status codes, and the
library stays usable afterwards.

* The reduction's grid barrier waits at most `reduce_spin_limit` polls; with
  a limit of 0 the first wait of a multi-CTA reduction gives up at once.  The
  kernel records PH0_ETIMEOUT, every CTA returns, and ph0_finish reports it;
  the same workspace then computes the oracle's bars.
* A serving context whose arena cannot be allocated returns PH0_ECUDA from
  ph0_ctx_create (nothing else is left allocated); a context that fits then
  works.
Bad arguments are rejected on the host (tests/test_capi_symbols.py)."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_reduction_wait_that_runs_out_reports_timeout_and_workspace_stays_usable():
    from paper_2203_02527_gb300 import ph0
    from paper_2203_02527_gb300._lib import Ph0Error
    x = inputs.uniform(4096, 3, seed=61)  # 64 reduction CTAs: some CTA always waits
    pts = torch.from_numpy(x).cuda()
    ws = ph0.Workspace(4096, 3)
    with pytest.raises(Ph0Error) as e:
        ph0.barcodes(pts, ws=ws, tuning={"reduce_spin_limit": 0})
    assert e.value.code == 5  # PH0_ETIMEOUT
    got = ph0.barcodes(pts, ws=ws)
    want, inf_v, nd = oracle.barcodes(x)
    assert_bars_equal(got.numpy(), want)
    assert got.stats["n_distinct"] == nd and got.inf[0] == inf_v
    # a limit that is never reached changes nothing
    again = ph0.barcodes(pts, ws=ws, tuning={"reduce_spin_limit": 1 << 20})
    assert_bars_equal(again.numpy(), want)


def test_serving_context_allocation_failure_is_reported():
    from paper_2203_02527_gb300._lib import Ph0Error
    from paper_2203_02527_gb300.serve import Server, run_stream
    with pytest.raises(Ph0Error) as e:
        Server(mem_budget=1 << 50)  # no GPU has a PiB of memory
    assert e.value.code == 6  # PH0_ECUDA
    x = inputs.uniform(300, 3, seed=62)
    with Server(mem_budget=1 << 28, streams=1) as srv:
        done = run_stream(srv, [x])
    assert done[0].status == 0
    assert_bars_equal(done[0].bars, oracle.barcodes(x)[0])
