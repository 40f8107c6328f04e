"""The autotuner's shape cache (host only): entries are keyed by GPU model, precision, transform
length and column bucket, survive a save/load round trip, and a name written by one GPU model is
never returned for another."""
import pytest

import paper_1501_01652_gb300 as hk


@pytest.fixture(autouse=True)
def _clean_cache():
    hk.tune_cache_clear()
    yield
    hk.tune_cache_clear()


def test_bucket_is_floor_log2_clamped():
    assert [hk.tune_bucket(n) for n in (1, 2, 3, 4, 7, 8, 64, 65, 1 << 20)] == [0, 1, 1, 2, 2, 3, 6, 6, 16]
    assert hk.tune_bucket(0) == 0


def test_keys_separate_gpu_models_and_fields(tmp_path):
    hk.tune_cache_put("NVIDIA GB300", "fp64", 21, 6, radices=[7, 7, 7], ms_default=10.0, ms_chosen=9.0)
    hk.tune_cache_put("NVIDIA GB300", "fp64", 21, 4, radices=[5, 8, 8])
    hk.tune_cache_put("NVIDIA GB300", "df64", 21, 6, radices=[5, 5, 5, 6])
    hk.tune_cache_put("Other GPU 2", "fp64", 21, 6, radices=[6, 7, 8])
    hk.tune_cache_put("NVIDIA GB300", "fp32", 11, 3, one_launch=True)
    assert hk.tune_cache_get("NVIDIA GB300", "fp64", 21, 6)["radices"] == [7, 7, 7]
    assert hk.tune_cache_get("NVIDIA GB300", "fp64", 21, 4)["radices"] == [5, 8, 8]
    assert hk.tune_cache_get("NVIDIA GB300", "df64", 21, 6)["radices"] == [5, 5, 5, 6]
    assert hk.tune_cache_get("Other GPU 2", "fp64", 21, 6)["radices"] == [6, 7, 8]
    assert hk.tune_cache_get("NVIDIA GB300", "fp32", 11, 3)["one_launch"]
    assert hk.tune_cache_get("NVIDIA GB300", "fp64", 20, 6) is None
    assert hk.tune_cache_get("NVIDIA GB30", "fp64", 21, 6) is None
    # a later store replaces its key only
    hk.tune_cache_put("NVIDIA GB300", "fp64", 21, 6, radices=[6, 7, 8])
    assert hk.tune_cache_get("NVIDIA GB300", "fp64", 21, 6)["radices"] == [6, 7, 8]
    assert hk.tune_cache_get("Other GPU 2", "fp64", 21, 6)["radices"] == [6, 7, 8]
    # save, clear, load
    path = tmp_path / "tune.txt"
    hk.tune_cache_save(path)
    hk.tune_cache_clear()
    assert hk.tune_cache_get("NVIDIA GB300", "fp64", 21, 4) is None
    hk.tune_cache_load(path)
    got = hk.tune_cache_get("NVIDIA GB300", "fp64", 21, 4)
    assert got["radices"] == [5, 8, 8] and got["precision"] == 1
    assert hk.tune_cache_get("NVIDIA GB300", "df64", 21, 6)["radices"] == [5, 5, 5, 6]
    assert hk.tune_cache_get("Other GPU 2", "fp64", 21, 6)["radices"] == [6, 7, 8]


def test_rejects_bad_names(tmp_path):
    with pytest.raises(RuntimeError, match="EINVAL"):
        hk.tune_cache_put("", "fp64", 21, 6, radices=[7, 7, 7])
    with pytest.raises(RuntimeError, match="EINVAL"):
        hk.tune_cache_put("two\nlines", "fp64", 21, 6, radices=[7, 7, 7])
    with pytest.raises(RuntimeError, match="EINVAL"):
        hk.tune_cache_load(tmp_path / "missing.txt")


def test_host_only_plans_report_no_shapes():
    p = hk.Plan("dht", 0, 4096, 1e-8, host_only=True)
    assert p.fft_shapes() == []
    assert p.info["fft_shapes"] == 0
