"""Host-side parts of the launch-shape autotuner: cache keys, the JSON cache
(atomic writes, unreadable files ignored) and the candidate list."""
import json

from paper_2011_00459_gb300 import autotune as A


def test_shape_keys_round_to_two_digits():
    assert A._round2(0) == 0
    assert A._round2(1_825_197) == 1_800_000
    assert A._round2(3_232_776.5) == 3_200_000
    assert A._round2(97) == 97
    k1 = A.shape_key("GB300", 1_000_000, 1)
    assert k1 == A.shape_key("GB300", 1_004_000, 1)
    assert k1 != A.shape_key("GB300", 1_000_000, 256)
    assert k1 != A.shape_key("GB300", 1_200_000, 1)
    assert k1 != A.shape_key("B200", 1_000_000, 1)


def test_cache_round_trip_and_bad_files(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "tune.json")
    monkeypatch.setenv(A.CACHE_ENV, path)
    assert A.cache_path() == path
    assert A.load_cache() == {}
    A.store_cache("k1", {"shape": {"pgs_blocks": 152, "pgs_sync": 1, "colour_blocks": 304, "pgs_threads": 768,
                                   "pgs_per_thread": 1}, "ms": 1.0})
    A.store_cache("k2", {"shape": {"pgs_blocks": 114, "pgs_sync": 0, "colour_blocks": 152}, "ms": 2.0})
    data = A.load_cache()
    assert set(data) == {"k1", "k2"} and data["k2"]["shape"]["pgs_sync"] == 0
    assert json.load(open(path)) == data
    open(path, "w").write("{not json")
    assert A.load_cache() == {}
    A.store_cache("k3", {"shape": {}, "ms": 3.0})  # rewrites a readable file
    assert list(A.load_cache()) == ["k3"]


def test_candidates_start_with_the_defaults_and_stay_in_limits():
    cfg = {"pgs_blocks": 304, "pgs_sync": 1, "colour_blocks": 608, "max_pgs_blocks": 304,
           "max_colour_blocks": 1216, "pgs_threads": 416, "pgs_per_thread": 1}
    c = A.candidates(cfg, 152)
    assert c[0] == {k: cfg[k] for k in A.KEYS}
    assert len(c) == len({tuple(sorted(x.items())) for x in c})
    per_sm = {(t, p): k for t, p, k in A.SHAPES}
    for x in c:
        assert x["colour_blocks"] == 608 and x["pgs_sync"] in (0, 1)
        # every shape gets the whole machine: 152 SMs x its CTAs per SM
        assert x["pgs_blocks"] == 152 * per_sm[(x["pgs_threads"], x["pgs_per_thread"])]
    assert {x["pgs_sync"] for x in c} == {0, 1}
    assert {(x["pgs_threads"], x["pgs_per_thread"]) for x in c} == set(per_sm)
    best = c[-1]
    bc = A.block_candidates(cfg, best)
    assert len(bc) == 1 and bc[0]["pgs_blocks"] == (3 * best["pgs_blocks"]) // 4
    assert dict(bc[0], pgs_blocks=best["pgs_blocks"]) == best
    cc = A.colour_candidates(cfg, best, 152)
    assert cc and all(dict(x, colour_blocks=best["colour_blocks"]) == best for x in cc)
    assert all(1 <= x["colour_blocks"] <= 1216 and x["colour_blocks"] != best["colour_blocks"] for x in cc)
    assert len(c) + len(bc) + len(cc) <= 18  # the tuner times them inside a settle reserve of 80 steps
    small = A.candidates(dict(cfg, pgs_blocks=3, pgs_sync=0), 152)
    assert all(x["pgs_blocks"] == max(1, 3 * per_sm[(x["pgs_threads"], x["pgs_per_thread"])] // 2) for x in small)
    assert A.block_candidates(dict(cfg, pgs_blocks=1), dict(small[0], pgs_blocks=1)) == []
