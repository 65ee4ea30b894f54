"""Host logic of the launch-shape autotuner: candidate list, cache keys and the
on-disk cache (no GPU needed)."""
import json
import os

from paper_2011_00162_gb300 import autotune


def test_candidates_cover_every_cap_of_every_variant():
    assert autotune.candidates({0: 2, 1: 3}) == [(0, 2), (0, 1), (1, 3), (1, 2), (1, 1)]
    assert autotune.candidates({0: 1}) == [(0, 1)]
    assert autotune.candidates({0: 0, 1: 1}) == [(0, 1), (1, 1)]  # at least one block per SM


def test_keys_separate_workloads():
    tag = "GPU|cc103|sm152"
    k = autotune.make_key(tag, 64, 841, 16, False)
    assert k != autotune.make_key(tag, 64, 841, 16, True)
    assert k != autotune.make_key(tag, 32, 841, 16, False)
    assert k != autotune.make_key(tag, 64, 840, 16, False)
    assert k != autotune.make_key(tag, 64, 841, 9, False)
    assert k != autotune.make_key("GPU|cc100|sm148", 64, 841, 16, False)
    assert k != autotune.make_key(tag, 64, 841, 16, False, kind="batch2m64")


def test_cache_round_trip_and_bad_files(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "cache.json")
    assert autotune.load_cache(path) == {}
    autotune.store_cache("a", {"variant": 1, "blocks_per_sm": 2}, path)
    autotune.store_cache("b", {"variant": 0, "blocks_per_sm": 1}, path)
    assert autotune.load_cache(path) == {"a": {"variant": 1, "blocks_per_sm": 2},
                                         "b": {"variant": 0, "blocks_per_sm": 1}}
    assert [f for f in os.listdir(tmp_path / "sub") if f.startswith(".autotune.")] == []
    # unreadable, foreign or old-version files read as empty and are replaced on the next store
    for bad in ["{not json", json.dumps([1, 2]), json.dumps({"version": 0, "entries": {"x": {}}})]:
        with open(path, "w") as fh:
            fh.write(bad)
        assert autotune.load_cache(path) == {}
    autotune.store_cache("c", {"variant": 0, "blocks_per_sm": 3}, path)
    assert list(autotune.load_cache(path)) == ["c"]
    # the environment variable chooses the default location
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "env.json"))
    assert autotune.cache_path() == str(tmp_path / "env.json")
    monkeypatch.delenv(autotune.CACHE_ENV)
    assert autotune.cache_path().endswith(os.path.join(".cache", "od2p", "autotune.json"))
