"""Host logic of the autotuning cache (no GPU): keys and the JSON round trip."""
import json

from paper_1605_02669_gb300 import acs, tuning


def test_shape_key_buckets_sizes_and_separates_memories():
    p = acs.params(m=64, memory=acs.ACS_MEM_MATRIX)
    a = tuning.shape_key([1002, 2392], p)
    # same power-of-two buckets -> same key; order does not matter
    assert tuning.shape_key([2392, 1010], p) == a
    assert tuning.shape_key([1002, 4100], p) != a
    q = acs.params(m=64, memory=acs.ACS_MEM_SPM, spm_slots=8)
    assert tuning.shape_key([1002, 2392], q) != a
    assert tuning.shape_key([1002, 2392], acs.params(m=128)) != a
    assert "B2" in a and "m64" in a


def test_cache_round_trip_and_corrupt_file(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tuning.load_cache(path) == {}
    tuning.save_cache(path, {"k": {"threads_per_ant": 32, "cluster_size": 16, "resident": 1}})
    assert tuning.load_cache(path)["k"]["cluster_size"] == 16
    with open(path, "w") as f:
        f.write("{not json")
    assert tuning.load_cache(path) == {}
    with open(path, "w") as f:
        json.dump([1, 2], f)
    assert tuning.load_cache(path) == {}
