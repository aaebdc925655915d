"""The autotuner's cache (host logic, no GPU): dimension and cloud-size
buckets, and a stored choice is found again for every cloud of the same
buckets on the same GPU name, and only there."""
import pytest

from paper_2203_02527_gb300 import autotune


@pytest.fixture
def fresh_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("PH0_TUNING_CACHE", str(tmp_path / "tuning.json"))
    monkeypatch.setattr(autotune, "_cache", None)
    monkeypatch.setattr(autotune, "_device_key", lambda: "GPU_A")
    yield tmp_path / "tuning.json"
    autotune._cache = None


def test_buckets():
    assert [autotune.bucket(d) for d in (1, 2, 3, 5, 16, 17, 33, 2000)] == [1, 2, 3, 8, 16, 32, 64, 1024]
    assert [autotune.n_bucket(n) for n in (2, 2048, 2049, 8192, 24576, 32768, 65535, 10**6)] == \
        [2048, 2048, 8192, 8192, 24576, 65535, 65535, 65535]


def test_store_and_lookup(fresh_cache, monkeypatch):
    choice = {"dist_split16": 16, "dist_tile": 128, "sort_top_bits": 9}
    assert autotune.cached(16, 32768) is None
    autotune._store(16, 32768, choice)
    assert fresh_cache.exists()
    assert autotune.cached(16, 30000) == choice      # same buckets
    assert autotune.cached(9, 65535) == choice       # d 9..16 share a bucket
    assert autotune.cached(16, 8192) is None         # another size bucket
    assert autotune.cached(3, 32768) is None         # another dimension bucket
    # read back from the file by a fresh process state
    monkeypatch.setattr(autotune, "_cache", None)
    assert autotune.cached(16, 32768) == choice
    # another GPU name misses
    monkeypatch.setattr(autotune, "_device_key", lambda: "GPU_B")
    assert autotune.cached(16, 32768) is None
