"""The autotuner's result cache (host logic of the binding; no GPU needed)."""
import json

import paper_1501_04706_gb300 as qh


def test_key_names_gpu_build_and_configuration():
    k = qh.tune_cache_key("NVIDIA GB300", (10, 3), qh.MODE_CHORD | qh.PREC_F64, 4096, 127_800_000)
    assert k.startswith("NVIDIA GB300|sm103|build=" + qh.library_build_id())
    assert "|flags=3|sets=4096|n=127800000" in k
    assert k != qh.tune_cache_key("NVIDIA GB300", (10, 3), qh.MODE_QUAD, 4096, 127_800_000)
    assert k != qh.tune_cache_key("NVIDIA B200", (10, 0), qh.MODE_CHORD | qh.PREC_F64, 4096, 127_800_000)


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert qh.tune_cache_load(path) == {}
    t1 = {"threads_per_block": 256, "items_per_thread": 16, "cutover": 4096, "grid_ctas_per_sm": 2, "cached": False}
    t2 = {"threads_per_block": 128, "items_per_thread": 8, "cutover": 2048, "grid_ctas_per_sm": 5}
    qh.tune_cache_store(path, "a", t1)
    qh.tune_cache_store(path, "b", t2)
    got = qh.tune_cache_load(path)
    assert got["a"] == {k: v for k, v in t1.items() if k != "cached"}
    assert got["b"] == t2
    with open(path) as f:
        assert json.load(f)["version"] == 1


def test_unreadable_file_is_an_empty_cache(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert qh.tune_cache_load(str(path)) == {}
    qh.tune_cache_store(str(path), "k", {"threads_per_block": 256, "items_per_thread": 8, "cutover": 3072,
                                         "grid_ctas_per_sm": 3})
    assert qh.tune_cache_load(str(path))["k"]["cutover"] == 3072
