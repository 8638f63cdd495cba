"""The autotuner: every candidate tiling renders the identical image; the
winner is one of them and is cached."""
import json

import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402
from paper_2311_16728_b300.autotune import CANDIDATES, autotune  # noqa: E402


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    base = S.tiny_scene(4096, seed=3)
    cam = S.tiny_camera()
    g = gsr.Gaussians.from_arrays(base.mean_op, base.quat, base.logscale, base.sh)
    vb = gsr.ViewBuffers(base.n, gsr.camera_from(cam), gsr.tiling_struct(16, 16), 1 << 16)
    vb.forward(g)
    gt = vb.img.clone()
    p = S.perturb(base)
    gp = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    before = [t.clone() for t in gp.tensors()]
    cache = tmp_path / "tiles.json"
    tile, report = autotune(gp, [(cam, gt)], steps=3, warmup=1, cache_path=str(cache))
    assert tuple(tile) in CANDIDATES
    assert all(report["identical_image"].values()) and len(report["ms_per_step"]) == len(CANDIDATES)
    assert all(torch.equal(a, b) for a, b in zip(before, gp.tensors()))  # caller's parameters untouched
    tile2, _ = autotune(gp, [(cam, gt)], cache_path=str(cache))
    assert tuple(tile2) == tuple(tile)
    assert json.load(open(cache))


def test_window_autotune_identical_views_and_cache(tmp_path):
    from paper_2311_16728_b300.autotune import WINDOW_CANDIDATES, autotune_window
    base = S.tiny_scene(4096, seed=3)
    cams = [S.tiny_camera(), S.pose_camera((0.1, 0.05, 0.0), 0.05, 150.0, 150.0, 160, 120)]
    g = gsr.Gaussians.from_arrays(base.mean_op, base.quat, base.logscale, base.sh)
    kf = []
    for cam in cams:
        vb = gsr.ViewBuffers(base.n, gsr.camera_from(cam), gsr.tiling_struct(16, 16), 1 << 16)
        vb.forward(g)
        kf.append((cam, vb.img.clone()))
    p = S.perturb(base)
    gp = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    before = [t.clone() for t in gp.tensors()]
    cache = tmp_path / "tiles.json"
    tile, report = autotune_window(gp, kf, steps=3, warmup=1, cache_path=str(cache))
    assert tuple(tile) in WINDOW_CANDIDATES
    assert all(report["identical_image"].values()) and len(report["ms_per_step"]) == len(WINDOW_CANDIDATES)
    assert all(torch.equal(a, b) for a, b in zip(before, gp.tensors()))
    tile2, _ = autotune_window(gp, kf, cache_path=str(cache))
    assert tuple(tile2) == tuple(tile)
