"""Serving and batching: the fused small-cloud kernel and the serving context
give, for every cloud, exactly the bars of the plain path (and of the
oracle), alone and in a mixed stream, under a memory budget that forces
admission to wait."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plain(x):
    from paper_2203_02527_gb300 import ph0
    return ph0.barcodes(torch.from_numpy(np.ascontiguousarray(x)).cuda()).numpy()


def _same(a, b):
    assert len(a) == len(b)
    assert a.tobytes() == b.tobytes()


def _mixed(count, seed, n_max=2000):
    rng = np.random.default_rng(seed)
    clouds = []
    for i in range(count):
        kind = i % 5
        n = int(rng.integers(2, 181)) if kind < 3 else int(rng.integers(181, n_max))
        d = int(rng.choice([1, 2, 3, 8, 32]))
        if i % 7 == 0:
            x = inputs.with_duplicates(n, d, max(1, n // 3), seed=seed + i)
        elif i % 11 == 0:
            x = inputs.lattice(int(np.ceil(n ** (1 / 2))), 2)[:n]
        else:
            x = inputs.gaussian_mixture(n, d, k=int(rng.integers(1, 6)), sigma=0.3, seed=seed + i)
        clouds.append(np.ascontiguousarray(x, np.float32))
    return clouds


def test_fused_small_batch_equals_plain_and_oracle():
    from paper_2203_02527_gb300.serve import Server, run_stream
    rng = np.random.default_rng(9)
    clouds = []
    for i in range(120):
        n = int(rng.integers(1, 181))
        d = int(rng.choice([1, 2, 3, 5, 16, 33, 64]))
        clouds.append(inputs.uniform(n, d, seed=500 + i) if i % 3 else inputs.negative_zero_mix(n, d, seed=i))
    with Server(mem_budget=1 << 30, streams=2, small_max_n=180, batch_max=64) as srv:
        done = run_stream(srv, clouds)
    for i, x in enumerate(clouds):
        f = done[i]
        assert f.status == 0
        assert f.inf_vertex == 0  # the bar that never dies, written by the fused kernel
        if len(x) > 1:
            _same(f.bars, _plain(x))
        if i % 10 == 0:
            want = oracle.barcodes(x)[0]
            assert f.bars.tobytes() == want.astype(f.bars.dtype).tobytes()


def test_mixed_stream_equals_plain_under_tight_budget():
    from paper_2203_02527_gb300 import ph0
    from paper_2203_02527_gb300.serve import Server, run_stream
    clouds = _mixed(60, seed=77)
    # room for only about two of the larger clouds at a time
    budget = 3 * max(ph0._lib.workspace_bytes(len(x), x.shape[1]) for x in clouds)
    with Server(mem_budget=budget, streams=4, small_max_n=180, batch_max=32) as srv:
        done = run_stream(srv, clouds)
    for i, x in enumerate(clouds):
        assert done[i].status == 0
        assert done[i].inf_vertex == 0
        _same(done[i].bars, _plain(x))


def _crowded(n, seed):
    # two clusters within 1e-12 of two points at distance 1: the cross
    # distances crowd into one long group of equal key >> 16 out of order, so
    # the fix-up asks for the complete sort
    rng = np.random.default_rng(seed)
    a = rng.random((n // 2, 3)) * 1e-12
    b = rng.random((n - n // 2, 3)) * 1e-12
    b[:, 1] = 1.0
    return np.ascontiguousarray(np.concatenate([a, b]), np.float32)


def test_served_crowded_clouds_run_again_with_the_complete_sort():
    """The serving context leaves the whole path's gated complete sort out and
    runs a cloud again in full when the fix-up flags it: clouds that need it,
    mixed with clouds that do not, still give exactly the plain path's bars
    (and the oracle's)."""
    from paper_2203_02527_gb300.serve import Server, run_stream
    clouds = []
    for i in range(24):
        clouds.append(_crowded(300 + 37 * i, seed=900 + i) if i % 2 == 0
                      else inputs.gaussian_mixture(250 + 41 * i, 3, k=3, sigma=0.3, seed=950 + i))
    with Server(mem_budget=4 << 30, streams=4, small_max_n=180, batch_max=32) as srv:
        done = run_stream(srv, clouds)
    for i, x in enumerate(clouds):
        assert done[i].status == 0
        _same(done[i].bars, _plain(x))
        if i % 6 == 0:
            want = oracle.barcodes(x)[0]
            assert done[i].bars.tobytes() == want.astype(done[i].bars.dtype).tobytes()


def _crowded_in(n, d, seed):
    # as _crowded, in d dimensions
    rng = np.random.default_rng(seed)
    a = rng.random((n // 2, d)) * 1e-12
    b = rng.random((n - n // 2, d)) * 1e-12
    b[:, 1] = 1.0
    return np.ascontiguousarray(np.concatenate([a, b]), np.float32)


def test_served_packed_clouds_equal_plain_and_the_oracle():
    """Clouds of 2,897 points and more in four or more dimensions take the
    packed sort, in the context as in plain calls; a crowded one (groups of
    more than 4096 equal key >> 22) is flagged by the packed fix-up and runs
    again in full.  Mixed with small clouds, each gives exactly the plain
    path's bars, and the oracle's."""
    from paper_2203_02527_gb300 import ph0
    from paper_2203_02527_gb300.serve import Server, run_stream
    clouds = [inputs.gaussian_mixture(2900 + 600 * i, (8, 16, 32)[i], k=3, sigma=0.3, seed=990 + i)
              for i in range(3)]
    clouds.append(_crowded_in(3000, 8, seed=993))
    clouds += [inputs.uniform(150 + 37 * i, 3, seed=994 + i) for i in range(6)]
    forms = [ph0.barcodes(torch.from_numpy(x).cuda()).stats["sort_form"] for x in clouds[:4]]
    assert forms == [1, 1, 1, 2]
    with Server(mem_budget=4 << 30, streams=4, small_max_n=180, batch_max=32) as srv:
        done = run_stream(srv, clouds)
    for i, x in enumerate(clouds):
        assert done[i].status == 0
        _same(done[i].bars, _plain(x))
    for i in (0, 3):
        want = oracle.barcodes(clouds[i])[0]
        assert done[i].bars.tobytes() == want.astype(done[i].bars.dtype).tobytes()


def test_serving_errors():
    from paper_2203_02527_gb300._lib import Ph0Error
    from paper_2203_02527_gb300.serve import Server
    with Server(mem_budget=2 << 20, host_budget=1 << 20, streams=1) as srv:
        big = inputs.uniform(20000, 3, seed=1)
        with pytest.raises(Ph0Error) as e:  # can never fit 2 MiB of device memory
            srv.submit(big, 1)
        assert e.value.code == 4
        x = inputs.uniform(50, 3, seed=2)
        assert srv.submit(x, 5) == 0
        with pytest.raises(Ph0Error):  # tag 5 still in use
            srv.submit(x, 5)
        got = []
        while not got:
            got = srv.poll(wait_ms=50)
        _same(got[0].bars, _plain(x))
