"""The JSON tuning cache of the binding (host logic, no GPU)."""
import json

from paper_2502_14148_gb300 import inputs, ocn


def test_cache_round_trip_and_keys(tmp_path):
    path = str(tmp_path / "t.json")
    assert ocn._tuning_cache(path, "a") is None                     # missing file reads as empty
    ocn._tuning_cache(path, "a", 4)
    ocn._tuning_cache(path, "b", [1, 2, 3])
    assert ocn._tuning_cache(path, "a") == 4 and ocn._tuning_cache(path, "b") == [1, 2, 3]
    assert json.load(open(path)) == {"a": 4, "b": [1, 2, 3]}
    (tmp_path / "bad.json").write_text("{not json")
    assert ocn._tuning_cache(str(tmp_path / "bad.json"), "a") is None   # a corrupt file reads as empty
    p = inputs.config("cbl_256")
    assert ocn.shape_key(p) == [256, 256, 128, 32, 5, "amd", 1]
    assert ocn.shape_key(dict(p, Nx=128)) != ocn.shape_key(p)
