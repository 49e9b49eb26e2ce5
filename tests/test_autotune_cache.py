"""Host logic of the tile autotuner (CPU): the JSON cache round trip, a
damaged cache file read as empty, a cached choice returned without timing
anything, and every candidate tile accepted by the rasterizer's argument
checks."""
import numpy as np
import pytest

from paper_2403_16862_gb300 import api, autotune, build, scenes


@pytest.fixture(scope="module")
def B():
    build.build()
    from paper_2403_16862_gb300 import _binding
    _binding.load()
    return _binding


def test_cache_round_trip_and_damaged_file(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("INPC_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}
    autotune._save({"a": [16, 8], "b:timings_ms": {"16x8": 1.5}})
    assert autotune._load() == {"a": [16, 8], "b:timings_ms": {"16x8": 1.5}}
    assert not any(p.name.startswith("tune.json.tmp") for p in path.parent.iterdir())
    path.write_text("{not json")
    assert autotune._load() == {}


def test_cached_choice_needs_no_timing(tmp_path, monkeypatch):
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "test device")
    cam = scenes.make_camera((0, 0, -3), 100, 100, 50, 40, 100, 80)
    opts = api.RasterOptions(n_channels=64, head_mode=True)

    class Pos:  # only the sample count is read before the cache lookup
        shape = (1234, 3)

    key = autotune.key_for(cam, opts, 1234)
    assert key == "100x80:n1234:F64:f32:test device"
    autotune._save({key: [32, 4]})
    assert autotune.tuned_tiles(cam, opts, None, Pos(), None, None) == (32, 4)


def test_candidates_pass_the_argument_checks(B):
    cam = api.camera(scenes.make_camera((0, 0, -3), 100, 100, 50, 40, 100, 80))
    sizes = []
    for tw, th in autotune.CANDIDATES:
        assert tw * th <= 256
        o = api.RasterOptions(n_channels=64, head_mode=True, tile_w=tw, tile_h=th).c()
        sizes.append(B.inpc_rasterize_workspace_size(cam, o, 5000))
    # the tile only regroups pixels: the workspace does not depend on it
    assert len(set(sizes)) == 1 and sizes[0] > 0
    assert len(set(autotune.CANDIDATES)) == len(autotune.CANDIDATES)
    assert np.all(np.array(autotune.CANDIDATES) > 0)
