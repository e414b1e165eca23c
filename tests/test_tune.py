"""Host-side logic of the autotuner's cache (no GPU): the key names what a
tuning depends on (the multiset of band limits and spins, precision,
recursion, real flag, device) and nothing else; the JSON-lines cache file
keeps one line per key, replaces a key's line on a second store, and stays
readable as JSON."""
import json

import pytest


@pytest.fixture(scope="module")
def mw():
    from paper_1110_6298_gb300 import build
    build.build()
    import paper_1110_6298_gb300.mw as m
    m.lib()
    return m


def test_key_is_a_multiset_and_names_its_inputs(mw):
    dev = "NVIDIA GB300"
    mixed = mw.PRECISIONS["mixed"]
    a = mw.tune_key([2048] * 16, [0] * 8 + [2] * 8, mixed, dev)
    b = mw.tune_key([2048] * 16, [2, 0] * 8, mixed, dev)
    assert a == b  # order of the maps does not matter
    assert "2048/0x8" in a and "2048/2x8" in a and "prec=1" in a and "delta=tn" in a and dev in a
    # graph capture does not change the work, so not the key
    assert mw.tune_key([2048] * 16, [0] * 8 + [2] * 8, mixed | mw.FLAG_GRAPH, dev) == a
    others = [mw.tune_key([2048] * 16, [0] * 16, mixed, dev),
              mw.tune_key([2048] * 15, [0] * 7 + [2] * 8, mixed, dev),
              mw.tune_key([1024] * 16, [0] * 8 + [2] * 8, mixed, dev),
              mw.tune_key([2048] * 16, [0] * 8 + [2] * 8, mw.PRECISIONS["mixed_tf32"], dev),
              mw.tune_key([2048] * 16, [0] * 8 + [2] * 8, mixed | mw.FLAG_DELTA_RISBO, dev),
              mw.tune_key([2048] * 16, [0] * 8 + [2] * 8, mixed, "another GPU")]
    assert len(set(others + [a])) == len(others) + 1
    # ragged plans: the multiset of (L, s)
    r1 = mw.tune_key([64, 512, 64], [1, 0, -2], mixed, dev)
    assert r1 == mw.tune_key([512, 64, 64], [0, -2, 1], mixed, dev)
    assert "64/-2x1" in r1 and "64/1x1" in r1 and "512/0x1" in r1
    # FP64 plans use Risbo's sweep whatever the flags say
    assert "delta=risbo" in mw.tune_key([32], [0], mw.PRECISIONS["fp64"], dev)
    with pytest.raises(mw.MWError):
        mw.tune_key([], [], mixed, dev)


def test_cache_store_lookup_replace(mw, tmp_path):
    path = tmp_path / "tune.jsonl"
    assert mw.tune_cache_lookup(path, "k1") is None  # no file yet
    mw.tune_cache_store(path, "k1", 512, 2, 256, 62.5)
    mw.tune_cache_store(path, "k2", 256, 1, 128, 10.25)
    assert mw.tune_cache_lookup(path, "k1") == {"chunk": 512, "groups": 2, "tn_threads": 256, "ms": 62.5}
    assert mw.tune_cache_lookup(path, "k2") == {"chunk": 256, "groups": 1, "tn_threads": 128, "ms": 10.25}
    mw.tune_cache_store(path, "k1", 128, 1, 256, 55.0)  # replaces k1's line
    assert mw.tune_cache_lookup(path, "k1") == {"chunk": 128, "groups": 1, "tn_threads": 256, "ms": 55.0}
    assert mw.tune_cache_lookup(path, "k3") is None
    lines = path.read_text().splitlines()
    assert len(lines) == 2
    recs = [json.loads(ln) for ln in lines]
    assert {r["key"] for r in recs} == {"k1", "k2"}
    # keys with a quote cannot be stored
    with pytest.raises(mw.MWError):
        mw.tune_cache_store(path, 'bad"key', 512, 2, 256)
    # a line of another writer's format is kept untouched
    path.write_text(path.read_text() + '{"key": "k9", "chunk": 256, "groups": 2, "tn_threads": 128, "ms": 1.0}\n')
    mw.tune_cache_store(path, "k2", 512, 2, 256, 9.0)
    assert mw.tune_cache_lookup(path, "k9")["chunk"] == 256
    assert len(path.read_text().splitlines()) == 3
