"""Autotuner host logic (CPU) and one tuning run on the GPU."""
import json

import numpy as np
import pytest

from paper_2505_18992_gb300 import autotune as at


def test_valid_tiles_follow_the_library_rules():
    assert at.valid_tile(8, 16) and at.valid_tile(16, 16) and at.valid_tile(32, 16)
    assert not at.valid_tile(3, 16)      # width not in {4, 8, 16, 32}
    assert not at.valid_tile(32, 32)     # 1024 threads per tile
    assert not at.valid_tile(8, 7)       # odd height
    assert not at.valid_tile(4, 8)       # 32 pixels: not a multiple of 64


def test_candidates_divide_the_views_and_drop_invalid_tiles():
    cs = at.candidates(8, tiles=((8, 16), (32, 32)), persistent=(0, 4))
    assert all(c.tile_w == 8 and c.tile_h == 16 for c in cs)
    assert sorted({c.views_per_call for c in cs}) == [1, 4, 8]
    assert len(cs) == 2 * 3
    assert {c.views_per_call for c in at.candidates(1)} == {1}


def test_workload_key_rounds_the_gaussian_count():
    assert at.workload_key(1_000_000, 1200, 680, 1) == "n1000000_1200x680_v1"
    assert at.workload_key(1_012_345, 1200, 680, 1) == "n1000000_1200x680_v1"
    assert at.workload_key(2_049_000, 640, 480, 8) == "n2000000_640x480_v8"
    assert at.workload_key(57, 10, 10, 1) == "n57_10x10_v1"


def test_pick_and_cache_roundtrip(tmp_path):
    a, b = at.LaunchShape(8, 16), at.LaunchShape(16, 16, 4, 2)
    assert at.pick({a: 2.0, b: 1.5}) == b
    with pytest.raises(ValueError):
        at.pick({})
    path = str(tmp_path / "tune.json")
    c = at.Cache(path)
    c.put("GPU X", "k1", b, 1.5)
    c2 = at.Cache(path)
    assert c2.get("GPU X", "k1") == (b, 1.5)
    assert c2.get("GPU X", "k2") is None and c2.get("GPU Y", "k1") is None
    json.loads(open(path).read())  # plain JSON on disk


def test_validation_rejects_changed_counts_images_or_list_positions():
    rng = np.random.default_rng(0)
    ref = {"rgb": rng.uniform(size=(1, 3, 4, 5)).astype(np.float32),
           "depth": rng.uniform(size=(1, 4, 5)).astype(np.float32),
           "alpha": rng.uniform(size=(1, 4, 5)).astype(np.float32),
           "t_final": rng.uniform(size=(1, 4, 5)).astype(np.float32),
           "n_contrib": rng.integers(0, 9, (1, 4, 5)).astype(np.int32),
           "n_iter": rng.integers(0, 20, (1, 4, 5)).astype(np.int32)}
    same = {k: v.copy() for k, v in ref.items()}
    assert at.compare_outputs(same, ref, ref) is None
    near = {k: v.copy() for k, v in ref.items()}
    near["rgb"] = near["rgb"] + np.float32(8e-6)  # within 1e-5
    near["n_iter"] = near["n_iter"] + 1            # another tile shape's list positions
    assert at.compare_outputs(near, ref) is None
    assert "n_iter" in at.compare_outputs(near, ref, ref)
    bad = {k: v.copy() for k, v in ref.items()}
    bad["n_contrib"][0, 2, 3] += 1
    assert "n_contrib" in at.compare_outputs(bad, ref)
    bad = {k: v.copy() for k, v in ref.items()}
    bad["depth"][0, 1, 1] += 2e-5
    assert "depth" in at.compare_outputs(bad, ref)
    bad["depth"][0, 1, 1] = np.nan
    assert "depth" in at.compare_outputs(bad, ref)


@pytest.mark.gpu
def test_tuning_picks_a_valid_shape_and_the_image_does_not_depend_on_it(tmp_path):
    import torch

    from paper_2505_18992_gb300 import scenes
    from paper_2505_18992_gb300.render import Renderer
    from tests.helpers import intrinsics, scene_tensors

    sc = scenes.random_gaussians(20000, 256, 192, 220.0, seed=3, scale_range=(0.01, 0.1), n_views=2)
    g, T = scene_tensors(sc)
    intr = intrinsics(sc)
    g_rgb = torch.full((2, 3, 192, 256), 1e-5, device="cuda")
    shapes = at.candidates(2, tiles=((8, 16), (16, 16)), persistent=(0, 2))
    best, timings, rejected = at.tune(g, T, intr, g_rgb, shapes=shapes, steps=2,
                                      cache_path=str(tmp_path / "t.json"), return_rejected=True)
    assert not rejected, rejected  # every launch shape renders this frame as the default does
    assert best in shapes and len(timings) == len(shapes)
    assert all(t > 0 for t in timings.values())
    # the tuned shape renders the same image as the default shape (up to the rounding
    # of tile-local pixel offsets)
    a = Renderer(intr, n_views=2).forward(*g, T)
    b = Renderer(intr, n_views=2, tile_w=best.tile_w, tile_h=best.tile_h,
                 persistent_ctas=best.persistent_ctas).forward(*g, T)
    for k in ("rgb", "depth", "alpha"):
        assert float((a[k] - b[k]).abs().max()) <= 1e-5, k
    assert float((a["n_contrib"] != b["n_contrib"]).float().mean()) < 1e-3
    # a second call is served from the cache
    best2, t2 = at.tune(g, T, intr, g_rgb, cache_path=str(tmp_path / "t.json"))
    assert best2 == best and len(t2) == 1
