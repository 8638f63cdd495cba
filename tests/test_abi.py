"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/gsr.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gsr():
    from paper_2311_16728_b300 import _build
    _build.build()
    import paper_2311_16728_b300 as pkg
    return pkg


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gsr_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported_and_bound(gsr):
    lib = ctypes.CDLL(gsr._lib.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
        assert name in gsr._lib.EXPORTED, f"{name} has no Python binding"


def test_version_and_last_error(gsr):
    assert gsr._lib.gsr_version().decode().startswith("gsr")
    assert isinstance(gsr._lib.gsr_last_error(), bytes)


def test_camera_at_level_matches_pyramid_intrinsics(gsr):
    import synthetic as S
    cam = S.replica_camera(3)
    c = gsr.camera_from(cam)
    for lvl in range(3):
        got = gsr.camera_at_level(c, lvl)
        ref = S.camera_at_level(cam, lvl)
        assert (got.width, got.height) == (ref.width, ref.height)
        assert got.fx == pytest.approx(ref.fx) and got.cx == pytest.approx(ref.cx)
        assert got.cy == pytest.approx(ref.cy) and got.fy == pytest.approx(ref.fy)
    assert [gsr.camera_at_level(c, l).width for l in range(3)] == [1200, 600, 300]
    assert [gsr.camera_at_level(c, l).height for l in range(3)] == [680, 340, 170]


def test_bad_arguments_are_rejected_on_the_host(gsr):
    L = gsr._lib
    cam = gsr.camera_struct(np.eye(3), np.zeros(3), 100, 100, 50, 40, 100, 80)
    good_tiling = gsr.tiling_struct(16, 16)
    g = L.gsr_gaussians(16, 16, 16, 16, 10, 3)
    proj = L.gsr_proj(16, 16, 16, 16)
    # NULL outputs
    rc = L.gsr_preprocess.raw(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(good_tiling), None, None, None)
    assert rc == L.GSR_ERR_INVALID_ARG
    g2d = L.gsr_grad2d(16, 16, 16)
    rc = L.gsr_pose_bwd.raw(ctypes.byref(g), ctypes.byref(proj), ctypes.byref(cam), ctypes.byref(good_tiling),
                            ctypes.byref(g2d), None, None)
    assert rc == L.GSR_ERR_INVALID_ARG and b"d_pose" in L.gsr_last_error()
    rc = L.gsr_pose_bwd.raw(ctypes.byref(g), ctypes.byref(proj), ctypes.byref(cam), ctypes.byref(good_tiling),
                            ctypes.byref(L.gsr_grad2d(16, 24, 16)), 16, None)
    assert rc == L.GSR_ERR_INVALID_ARG and b"aligned" in L.gsr_last_error()
    # spatial order: empty box axis, short workspace; permute: unaligned plane
    lo3, hi3 = (ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(1, 0, 1)
    rc = L.gsr_spatial_order.raw(ctypes.byref(g), lo3, hi3, 16, 16, 1 << 20, None)
    assert rc == L.GSR_ERR_INVALID_ARG and b"hi > lo" in L.gsr_last_error()
    hi3 = (ctypes.c_float * 3)(1, 1, 1)
    rc = L.gsr_spatial_order.raw(ctypes.byref(g), lo3, hi3, 16, 16, 8, None)
    assert rc == L.GSR_ERR_CAPACITY
    pb, pb_bad = L.gsr_param_buffers(16, 16, 16, 16), L.gsr_param_buffers(16, 20, 16, 16)
    rc = L.gsr_permute.raw(ctypes.byref(pb), ctypes.byref(pb_bad), 16, 10, None)
    assert rc == L.GSR_ERR_INVALID_ARG and b"aligned" in L.gsr_last_error()
    # unaligned parameter plane
    g_bad = L.gsr_gaussians(18, 16, 16, 16, 10, 3)
    rc = L.gsr_preprocess.raw(ctypes.byref(g_bad), ctypes.byref(cam), ctypes.byref(good_tiling), ctypes.byref(proj),
                              None, None)
    assert rc == L.GSR_ERR_INVALID_ARG and b"aligned" in L.gsr_last_error()
    # SH degree out of range
    g_deg = L.gsr_gaussians(16, 16, 16, 16, 10, 4)
    rc = L.gsr_preprocess.raw(ctypes.byref(g_deg), ctypes.byref(cam), ctypes.byref(good_tiling), ctypes.byref(proj),
                              None, None)
    assert rc == L.GSR_ERR_INVALID_ARG
    # tiling that is not a multiple of a warp
    bad_tiling = gsr.tiling_struct(5, 5)
    rc = L.gsr_preprocess.raw(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(bad_tiling), ctypes.byref(proj),
                              None, None)
    assert rc == L.GSR_ERR_INVALID_ARG
    # launch shapes: staging batch a multiple of 32 up to 512; backward
    # threads 0, two pixels a thread, or 64 for 16 x 16 tiles
    for bad in [(16, 16, 48, 0), (16, 16, 1024, 0), (16, 16, -32, 0), (32, 8, 0, 64), (16, 16, 0, 256)]:
        rc = L.gsr_preprocess.raw(ctypes.byref(g), ctypes.byref(cam), ctypes.byref(gsr.tiling_struct(*bad)),
                                  ctypes.byref(proj), None, None)
        assert rc == L.GSR_ERR_INVALID_ARG, bad
    sz = ctypes.c_size_t()
    for ok in [(16, 16, 32, 0), (16, 16, 512, 128), (16, 16, 0, 64), (32, 8, 256, 128), (8, 32, 64, 0)]:
        assert L.gsr_bin_sort_workspace_size.raw(10, 16, ctypes.byref(cam), ctypes.byref(gsr.tiling_struct(*ok)),
                                                 ctypes.byref(sz)) == 0, ok
    # workspace too small
    rc = L.gsr_bin_sort.raw(ctypes.byref(proj), 10, ctypes.byref(cam), ctypes.byref(good_tiling), 16, 16, 100, 16, 16,
                            16, 1, None, None)
    assert rc == L.GSR_ERR_CAPACITY
    # loss: lambda outside [0, 1]
    rc = L.gsr_loss_fwd_bwd.raw(16, 16, 3, 8, 8, ctypes.c_float(1.5), 16, 16, 16, 1 << 20, None)
    assert rc == L.GSR_ERR_INVALID_ARG


def test_workspace_queries(gsr):
    L = gsr._lib
    sz = ctypes.c_size_t()
    cam = gsr.camera_struct(np.eye(3), np.zeros(3), 600, 600, 600, 340, 1200, 680)
    t = gsr.tiling_struct(16, 16)
    L.gsr_bin_sort_workspace_size(300000, 2_000_000, ctypes.byref(cam), ctypes.byref(t), ctypes.byref(sz))
    assert sz.value >= 12 * 2_000_000
    L.gsr_loss_workspace_size(3, 680, 1200, ctypes.byref(sz))
    assert sz.value >= 3 * 3 * 680 * 1200 * 4


def test_defaults_match_paper_hyperparameters(gsr):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_hyperparameters.json")))
    assert gsr.LAMBDA_DSSIM == gold["lambda_dssim"]["value"]
    assert gsr.PYRAMID_LEVELS == gold["pyramid_levels"]["value"]
    assert 48 // 3 == gold["sh_coeffs_per_channel"]["value"]  # 12 float4 planes = 16 coefficients x RGB


def test_batched_arguments_are_rejected_on_the_host(gsr):
    L = gsr._lib
    cam = gsr.camera_struct(np.eye(3), np.zeros(3), 100, 100, 50, 40, 100, 80)
    sz = ctypes.c_size_t()
    cams65 = (L.gsr_camera * 65)(*([cam] * 65))
    assert L.gsr_batched_iterate_workspace_size.raw(cams65, 65, ctypes.byref(sz)) == L.GSR_ERR_INVALID_ARG
    assert L.gsr_batched_iterate_workspace_size.raw(cams65, 0, ctypes.byref(sz)) == L.GSR_ERR_INVALID_ARG
    assert L.gsr_batched_iterate_workspace_size.raw(cams65, 2, ctypes.byref(sz)) == L.GSR_OK
    # three SSIM maps of 3 x 100 x 80 per view, 2 partials per 32 x 32 block (4 x 3 blocks x 3 channels)
    assert sz.value >= 2 * (3 * 3 * 100 * 80 * 4 + 2 * 36 * 4)
    # the persistent kernel runs 256-pixel tiles only
    proj = L.gsr_proj(16, 16, 16, 16)
    g2 = L.gsr_grad2d(16, 16, 16)
    ptrs = (ctypes.c_void_p * 1)(16)
    rc = L.gsr_batched_iterate.raw(ctypes.byref(proj), None, 16, cams65, 1, ctypes.byref(gsr.tiling_struct(16, 8)),
                                   None, ptrs, ptrs, ptrs, ptrs, ptrs, None, 0.2, 16, ctypes.byref(g2), 16, 1 << 30,
                                   None, None)
    assert rc == L.GSR_ERR_UNSUPPORTED and b"256-pixel" in L.gsr_last_error()
    # lambda outside [0, 1]
    rc = L.gsr_batched_iterate.raw(ctypes.byref(proj), None, 16, cams65, 1, ctypes.byref(gsr.tiling_struct(16, 16)),
                                   None, ptrs, ptrs, ptrs, ptrs, ptrs, None, 1.5, 16, ctypes.byref(g2), 16, 1 << 30,
                                   None, None)
    assert rc == L.GSR_ERR_INVALID_ARG
    # too many views for the batched binning
    g = L.gsr_gaussians(16, 16, 16, 16, 10, 3)
    rc = L.gsr_batched_preprocess.raw(ctypes.byref(g), cams65, 65, ctypes.byref(gsr.tiling_struct(16, 16)),
                                      ctypes.byref(proj), None)
    assert rc == L.GSR_ERR_INVALID_ARG


def test_default_init_sizes_and_arguments(gsr):
    L = gsr._lib
    sz = ctypes.c_size_t()
    for M, n in ((0, 5000), (1, 1), (700, 20000), (20000, 500000)):
        assert L.gsr_default_init_workspace_size.raw(M, n, ctypes.byref(sz)) == L.GSR_OK
        assert sz.value >= 12 * M
    assert L.gsr_default_init_workspace_size.raw(-1, 10, ctypes.byref(sz)) == L.GSR_ERR_INVALID_ARG
    cam = gsr.camera_struct(np.eye(3), np.zeros(3), 100, 100, 50, 40, 100, 80)
    buf = L.gsr_param_buffers(16, 16, 16, 16)
    # slots beyond the map
    rc = L.gsr_default_init.raw(16, 100, 80, 16, 10, ctypes.byref(cam), ctypes.byref(buf), 5, 0, 16, 1 << 20, None)
    assert rc == L.GSR_ERR_INVALID_ARG


def test_build_script_loads_without_the_package():
    """build() compiles before anything imports the package (whose import
    fails loudly without the library): its build script loads by path alone."""
    import subprocess
    import sys
    code = ("import importlib.util, os, sys; root = os.getcwd(); "
            "spec = importlib.util.spec_from_file_location('gsr_build', "
            "os.path.join(root, 'paper_2311_16728_b300', '_build.py')); "
            "mod = importlib.util.module_from_spec(spec); spec.loader.exec_module(mod); "
            "assert callable(mod.build) and mod.sources(); "
            "assert 'paper_2311_16728_b300' not in sys.modules")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_autotune_driver_rejects_bad_arguments(gsr):
    """Checked before any CUDA call: no candidates, no callback, no steps."""
    L = gsr._lib
    fn = L.AUTOTUNE_FN(lambda c, a, ctx: 0)
    ms = (ctypes.c_float * 2)()
    best = ctypes.c_int32(7)
    assert L.gsr_autotune.raw(0, fn, None, 1, 1, None, ms, ctypes.byref(best)) == L.GSR_ERR_INVALID_ARG
    assert L.gsr_autotune.raw(2, L.AUTOTUNE_FN(), None, 1, 1, None, ms, ctypes.byref(best)) == L.GSR_ERR_INVALID_ARG
    assert L.gsr_autotune.raw(2, fn, None, 1, 0, None, ms, ctypes.byref(best)) == L.GSR_ERR_INVALID_ARG
    assert b"gsr_autotune" in L.gsr_last_error()
