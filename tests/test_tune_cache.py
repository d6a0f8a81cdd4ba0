"""The autotuner's file cache on the host (no device work): entries stored
under a key come back unchanged, other keys survive a store, a file that is
not a cache is never overwritten, and bad keys are rejected."""
import json

import pytest

from paper_1804_08487_gb300 import build, cb

S1 = {"tile_max": 32, "block_max": 2048, "smem_max": 4096, "inorder_threads": 256, "retry_passes": 2}
S2 = {"tile_max": 128, "block_max": 512, "smem_max": 8192, "inorder_threads": 1024, "retry_passes": 0}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build_cuda()
    return cb.load()


def test_missing_file_is_an_empty_cache(tmp_path):
    assert cb.cb_tune_cache_lookup(str(tmp_path / "none.json"), "GB300|sm152|n25|g0|0,1") is None


def test_store_then_lookup_and_keep_other_keys(tmp_path):
    p = str(tmp_path / "tune.json")
    cb.cb_tune_cache_store(p, "a|1", S1)
    cb.cb_tune_cache_store(p, "b|2", S2)
    assert cb.cb_tune_cache_lookup(p, "a|1") == S1
    assert cb.cb_tune_cache_lookup(p, "b|2") == S2
    assert cb.cb_tune_cache_lookup(p, "a|") is None            # no prefix match
    # replacing one key keeps the other and leaves one entry per key
    cb.cb_tune_cache_store(p, "a|1", S2)
    assert cb.cb_tune_cache_lookup(p, "a|1") == S2
    assert cb.cb_tune_cache_lookup(p, "b|2") == S2
    doc = json.loads(open(p).read())                           # the file is valid JSON
    assert doc["version"] == 1
    assert sorted(e["key"] for e in doc["entries"]) == ["a|1", "b|2"]
    assert not (tmp_path / "tune.json.tmp").exists()


def test_foreign_file_is_left_alone(tmp_path):
    p = tmp_path / "notes.json"
    p.write_text('{"something": "else"}\n')
    with pytest.raises(cb.CbError) as e:
        cb.cb_tune_cache_store(str(p), "a|1", S1)
    assert e.value.code == cb.CB_EIO
    with pytest.raises(cb.CbError) as e:
        cb.cb_tune_cache_lookup(str(p), "a|1")
    assert e.value.code == cb.CB_EIO
    assert p.read_text() == '{"something": "else"}\n'


def test_malformed_entry_is_an_error(tmp_path):
    p = tmp_path / "tune.json"
    p.write_text('{"version": 1, "entries": [\n    {"key": "a|1", "tile_max": 32}\n]}\n')
    with pytest.raises(cb.CbError) as e:
        cb.cb_tune_cache_lookup(str(p), "a|1")
    assert e.value.code == cb.CB_EIO
    # a store drops the malformed entry it cannot read and keeps the file a cache
    cb.cb_tune_cache_store(str(p), "b|2", S1)
    assert cb.cb_tune_cache_lookup(str(p), "b|2") == S1


@pytest.mark.parametrize("key", ["", 'a"b', "a\\b", "a{b", "a}b", "a\nb"])
def test_bad_keys_are_rejected(tmp_path, key):
    with pytest.raises(cb.CbError) as e:
        cb.cb_tune_cache_store(str(tmp_path / "t.json"), key, S1)
    assert e.value.code == cb.CB_EINVAL


def test_unwritable_path_is_an_io_error(tmp_path):
    with pytest.raises(cb.CbError) as e:
        cb.cb_tune_cache_store(str(tmp_path / "no_dir" / "t.json"), "a|1", S1)
    assert e.value.code == cb.CB_EIO
