"""Autotuner for the screen tiling and launch shape of the mapping iteration.

The rendered image does not depend on the tiling (each Gaussian reaches only
its own pixel box, and the tile cull never drops a pair that blends) nor on
the blend kernels' launch shape, so all three knobs are pure performance
choices: the tile shape, the staging batch depth (depth-ordered records
staged in shared memory per round: 32 .. 256 for the whole tile, or 0 =
every warp its own 32 for 16 x 16 tiles, one per thread otherwise) and the
backward blend's threads per tile (for 16 x 16 tiles: 64 threads of four
pixels, or 128 of two).  The tuner times a few captured iterations of every
(tile, depth, threads) candidate on the caller's workload (the library's
timing driver, gsr_autotune, calls back to set up, step and release each
candidate and times the steps with CUDA events), checks that every candidate
renders a bit-identical image, and caches the winner per (GPU, width,
height, Gaussian-count bucket).
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional, Sequence, Tuple

import ctypes

import torch

from . import _lib as L
from .raster import Gaussians, MappingStep, ViewBuffers, camera_from, ensure_capacity, tiling_struct

# (tile_w, tile_h): every shape the blend kernels accept with 64..512 threads
TILES: Tuple[Tuple[int, int], ...] = ((16, 16), (32, 8), (8, 32), (16, 8), (32, 16), (16, 32), (32, 32))
# staging batch depths (0: warp-private for 16 x 16 tiles, else one record per thread)
DEPTHS: Tuple[int, ...] = (0, 32, 64, 128, 256)


def grid(tiles: Sequence[Tuple[int, int]], depths: Sequence[int] = DEPTHS) -> Tuple[Tuple[int, int, int, int], ...]:
    """(tile_w, tile_h, batch_depth, bwd_threads) candidates: every tile x
    depth, and for 16 x 16 tiles both backward launch shapes (0 = 64 threads
    of four pixels, 128 = two pixels a thread)."""
    out = []
    for tw, th in tiles:
        for d in depths:
            for bt in ((0, 128) if (tw, th) == (16, 16) else (0,)):
                out.append((tw, th, d, bt))
    return tuple(out)


def label(c) -> str:
    tw, th, d, bt = c
    dl = d or ("W" if (tw, th) == (16, 16) else "T")  # W: warp-private staging, T: one record per thread
    return f"{tw}x{th}/depth{dl}/bwd{bt or 'default'}"


CANDIDATES = grid(TILES)


def _key(width: int, height: int, n: int) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{dev}|{width}x{height}|n2^{max(0, math.ceil(math.log2(max(n, 1))))}"


def _clone(g: Gaussians) -> Gaussians:
    return Gaussians(*(t.clone() for t in g.tensors()), g.sh_degree)


def _tune(n: int, setup, step, release, warmup: int, steps: int):
    """Times candidates 0 .. n-1 with the native driver (gsr_autotune) on the
    current stream; setup / step / release(c) are called back for candidate
    c.  Returns (median ms per candidate, index of the fastest)."""
    errors = []

    def callback(c, action, _ctx):
        try:
            (setup, step, release)[action](c)
            return 0
        except BaseException as e:  # re-raised below, after the driver returns
            errors.append(e)
            return L.GSR_ERR_INVALID_ARG

    fn = L.AUTOTUNE_FN(callback)
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int32(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.gsr_autotune.raw(n, fn, None, warmup, steps, stream, ms, ctypes.byref(best))
    if errors:
        raise errors[0]
    if rc != 0:
        raise RuntimeError(f"gsr_autotune: {L.gsr_last_error().decode()}")
    return [float(v) for v in ms], int(best.value)


def autotune(params: Gaussians, views: Sequence, candidates: Sequence[Tuple[int, int, int, int]] = CANDIDATES,
             steps: int = 10, warmup: int = 3, cache_path: Optional[str] = None, verbose: bool = False):
    """Returns ((tile_w, tile_h, batch_depth, bwd_threads), report).  `views` =
    [(camera, gt image)] as for MappingStep; the caller's parameters are not
    modified."""
    cam0 = camera_from(views[0][0])
    key = _key(cam0.width, cam0.height, params.n)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return tuple(cache[key]["tile"]), cache[key]
    report = {"key": key, "ms_per_step": {}, "identical_image": {}}
    state = {"ref": None, "ms": None}

    def setup(c):
        tiling = tiling_struct(*candidates[c])
        # image check on the first view, untouched parameters
        vb = ViewBuffers(params.n, cam0, tiling, 1024)
        ensure_capacity(vb, params)
        vb.forward(params)
        img = vb.img.clone()
        if state["ref"] is None:
            state["ref"] = img
        same = bool(torch.equal(img, state["ref"]))
        report["identical_image"][label(candidates[c])] = same
        if not same:
            raise RuntimeError(f"tiling {label(candidates[c])} changed the rendered image")
        del vb
        # timing on a copy of the parameters
        state["ms"] = MappingStep(_clone(params), views, tiling)
        state["ms"].capture()

    def release(c):
        state["ms"] = None

    times, best = _tune(len(candidates), setup, lambda c: state["ms"].step(), release, warmup, steps)
    for c, t in zip(candidates, times):
        report["ms_per_step"][label(c)] = t
        if verbose:
            print(f"autotune {label(c)}: {t:.4f} ms/step")
    tile = tuple(int(v) for v in candidates[best])
    report["tile"] = list(tile)
    report["chosen"] = label(tile)
    if cache_path:
        cache[key] = report
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return tile, report


# tile shapes the persistent window kernel accepts (256 pixels, 128 threads)
WINDOW_TILES: Tuple[Tuple[int, int], ...] = ((16, 16), (32, 8), (8, 32))
WINDOW_CANDIDATES = grid(WINDOW_TILES)


def autotune_window(params: Gaussians, keyframes: Sequence, levels: int = 3,
                    candidates: Sequence[Tuple[int, int, int, int]] = WINDOW_CANDIDATES, steps: int = 10,
                    warmup: int = 3, cache_path: Optional[str] = None, verbose: bool = False):
    """Tile shape, staging batch depth and backward threads per tile of the
    batched pyramid window: every candidate must render every view
    bit-identically; the fastest captured iteration wins.  Returns
    ((tile_w, tile_h, batch_depth, bwd_threads), report); the caller's
    parameters are not modified."""
    from .batched import BatchedWindow
    cam0 = camera_from(keyframes[0][0])
    key = "window|" + _key(cam0.width, cam0.height, params.n) + f"|kf{len(keyframes)}|l{levels}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return tuple(cache[key]["tile"]), cache[key]
    report = {"key": key, "ms_per_step": {}, "identical_image": {}}
    state = {"ref": None, "bw": None}

    def setup(c):
        bw = BatchedWindow(_clone(params), keyframes, levels=levels, tiling=tiling_struct(*candidates[c]))
        bw.preprocess()
        bw.bin_sort()
        bw.iterate()
        torch.cuda.synchronize()
        imgs = [t.clone() for t in bw.imgs]
        if state["ref"] is None:
            state["ref"] = imgs
        same = all(torch.equal(a, b) for a, b in zip(imgs, state["ref"]))
        report["identical_image"][label(candidates[c])] = same
        if not same:
            raise RuntimeError(f"tiling {label(candidates[c])} changed a rendered view")
        # the eager pass above left screen-space gradients behind: clear them
        bw.g2.zero_()
        bw.capture()
        state["bw"] = bw

    def release(c):
        bw, state["bw"] = state["bw"], None
        if bw is not None and bw.status.item() != 0:
            raise RuntimeError(f"tiling {label(candidates[c])}: device status {bw.status.item():#x}")

    times, best = _tune(len(candidates), setup, lambda c: state["bw"].step(), release, warmup, steps)
    for c, t in zip(candidates, times):
        report["ms_per_step"][label(c)] = t
        if verbose:
            print(f"autotune window {label(c)}: {t:.4f} ms/step")
    tile = tuple(int(v) for v in candidates[best])
    report["tile"] = list(tile)
    report["chosen"] = label(tile)
    if cache_path:
        cache[key] = report
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return tile, report
