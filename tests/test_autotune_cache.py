"""The autotuner's cache file (igr.autotune_key / autotune_cache_*), without a GPU."""
import json
from dataclasses import replace

from paper_2505_07392_gb300 import igr, inputs


def test_key_separates_what_the_shape_depends_on():
    c = inputs.blast(32)
    k = igr.autotune_key(c, "f16", False, "GB300")
    others = [igr.autotune_key(c, "f32", False, "GB300"),
              igr.autotune_key(replace(c, nz=16), "f16", False, "GB300"),
              igr.autotune_key(replace(c, order=3), "f16", False, "GB300"),
              igr.autotune_key(replace(c, sigma_solver=1), "f16", False, "GB300"),
              igr.autotune_key(replace(c, mu=1e-3), "f16", False, "GB300"),
              igr.autotune_key(c, "f16", True, "GB300"),
              igr.autotune_key(c, "f16", False, "another GPU")]
    assert len(set(others + [k])) == len(others) + 1
    # boundary kinds and jets change nothing the shape depends on
    assert igr.autotune_key(replace(c, bc=(0,) * 6), "f16", False, "GB300") == k


def test_store_and_load(tmp_path):
    p = str(tmp_path / "tiles.json")
    assert igr.autotune_cache_load(p) == {}
    igr.autotune_cache_store(p, "a", {"tiles": [8, 8, 32], "forms": [1, 0]})
    igr.autotune_cache_store(p, "b", {"tiles": [4, 4, 4], "forms": [0, 0]})
    d = igr.autotune_cache_load(p)
    assert d == {"a": {"tiles": [8, 8, 32], "forms": [1, 0]}, "b": {"tiles": [4, 4, 4], "forms": [0, 0]}}
    assert not [f for f in tmp_path.iterdir() if ".tmp" in f.name]
    (tmp_path / "bad.json").write_text("{not json")
    assert igr.autotune_cache_load(str(tmp_path / "bad.json")) == {}
    assert json.load(open(p))["a"]["tiles"] == [8, 8, 32]
