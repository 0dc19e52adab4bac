"""Host side of the batch autotune cache: the key and the JSON file."""
import json
import types

from paper_2503_16422_gb300 import fdgs


def _cam(w, h):
    return types.SimpleNamespace(width=w, height=h)


def test_key_buckets_sizes_by_tile_grid_and_scene_by_power_of_two():
    a = fdgs.autotune_key([_cam(1352, 1014), _cam(1352, 1014)], 200_000, True, (0, 0, 0), "G")
    # same 16x16 tile grids (85x64), same power-of-two bucket, order of requests irrelevant
    b = fdgs.autotune_key([_cam(1350, 1009), _cam(1345, 1012)], 150_000, True, (0, 0, 0), "G")
    assert a == b
    assert "tiles=85x64*2" in a and "gauss<=262144" in a
    assert a != fdgs.autotune_key([_cam(1352, 1014)] * 2, 300_000, True, (0, 0, 0), "G")
    assert a != fdgs.autotune_key([_cam(1352, 1014)] * 3, 200_000, True, (0, 0, 0), "G")
    assert a != fdgs.autotune_key([_cam(1352, 1014)] * 2, 200_000, False, (0, 0, 0), "G")
    assert a != fdgs.autotune_key([_cam(1352, 1014)] * 2, 200_000, True, (0.1, 0, 0), "G")
    assert a != fdgs.autotune_key([_cam(1352, 1014)] * 2, 200_000, True, (0, 0, 0), "H")
    mixed = fdgs.autotune_key([_cam(16, 16), _cam(512, 512), _cam(17, 16)], 1, True, (0,) * 3, "G")
    assert "tiles=1x1*1,2x1*1,32x32*1" in mixed and "gauss<=1" in mixed


def test_cache_file_roundtrip_and_bad_files(tmp_path):
    path = str(tmp_path / "c.json")
    assert fdgs.read_autotune_cache(path) == {}
    fdgs.write_autotune_cache(path, "k1", 6, 24)
    fdgs.write_autotune_cache(path, "k2", 5, 7)
    fdgs.write_autotune_cache(path, "k1", 4, 12)
    assert fdgs.read_autotune_cache(path) == {"k1": {"footprint": 4, "ctas_per_sm": 12},
                                              "k2": {"footprint": 5, "ctas_per_sm": 7}}
    with open(path, "w") as f:
        f.write("{not json")
    assert fdgs.read_autotune_cache(path) == {}
    with open(path, "w") as f:
        json.dump([1, 2], f)
    assert fdgs.read_autotune_cache(path) == {}
