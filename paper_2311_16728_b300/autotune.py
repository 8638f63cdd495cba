"""Autotuner for the screen tiling of the mapping iteration.

The rendered image does not depend on the tiling (each Gaussian reaches only
its own pixel box, and the tile cull never drops a pair that blends), so the
tile shape -- which also fixes the staging batch (one record per thread per
batch) and the threads per tile (one per two pixels) -- is a pure performance
choice.  The tuner times a few captured iterations of each candidate on the
caller's workload, checks that every candidate renders a bit-identical image,
and caches the winner per (GPU, width, height, Gaussian-count bucket).
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Optional, Sequence, Tuple

import torch

from .raster import Gaussians, MappingStep, ViewBuffers, camera_from, ensure_capacity, tiling_struct

# (tile_w, tile_h): every shape the blend kernels accept with 64..512 threads
CANDIDATES: Tuple[Tuple[int, int], ...] = ((16, 16), (32, 8), (8, 32), (16, 8), (32, 16), (16, 32), (32, 32))


def _key(width: int, height: int, n: int) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{dev}|{width}x{height}|n2^{max(0, math.ceil(math.log2(max(n, 1))))}"


def _clone(g: Gaussians) -> Gaussians:
    return Gaussians(*(t.clone() for t in g.tensors()), g.sh_degree)


def autotune(params: Gaussians, views: Sequence, candidates: Sequence[Tuple[int, int]] = CANDIDATES,
             steps: int = 10, warmup: int = 3, cache_path: Optional[str] = None, verbose: bool = False):
    """Returns ((tile_w, tile_h), report).  `views` = [(camera, gt image)] as for
    MappingStep; the caller's parameters are not modified."""
    cam0 = camera_from(views[0][0])
    key = _key(cam0.width, cam0.height, params.n)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return tuple(cache[key]["tile"]), cache[key]
    ref_img = None
    report = {"key": key, "ms_per_step": {}, "identical_image": {}}
    for tw, th in candidates:
        tiling = tiling_struct(tw, th)
        # image check on the first view, untouched parameters
        vb = ViewBuffers(params.n, cam0, tiling, 1024)
        ensure_capacity(vb, params)
        vb.forward(params)
        img = vb.img.clone()
        if ref_img is None:
            ref_img = img
        same = bool(torch.equal(img, ref_img))
        report["identical_image"][f"{tw}x{th}"] = same
        if not same:
            raise RuntimeError(f"tiling {tw}x{th} changed the rendered image")
        del vb
        # timing on a copy of the parameters
        ms = MappingStep(_clone(params), views, tiling)
        ms.capture()
        for _ in range(warmup):
            ms.step()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ms.step()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        report["ms_per_step"][f"{tw}x{th}"] = statistics.median(times)
        if verbose:
            print(f"autotune {tw}x{th}: {report['ms_per_step'][f'{tw}x{th}']:.4f} ms/step")
        del ms
    best = min(report["ms_per_step"], key=report["ms_per_step"].get)
    tile = tuple(int(v) for v in best.split("x"))
    report["tile"] = list(tile)
    if cache_path:
        cache[key] = report
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return tile, report


# tile shapes the persistent window kernel accepts (256 pixels, 128 threads)
WINDOW_CANDIDATES: Tuple[Tuple[int, int], ...] = ((16, 16), (32, 8), (8, 32))


def autotune_window(params: Gaussians, keyframes: Sequence, levels: int = 3,
                    candidates: Sequence[Tuple[int, int]] = WINDOW_CANDIDATES, steps: int = 10, warmup: int = 3,
                    cache_path: Optional[str] = None, verbose: bool = False):
    """Tile shape of the batched pyramid window: every candidate must render
    every view bit-identically; the fastest captured iteration wins.  Returns
    ((tile_w, tile_h), report); the caller's parameters are not modified."""
    from .batched import BatchedWindow
    cam0 = camera_from(keyframes[0][0])
    key = "window|" + _key(cam0.width, cam0.height, params.n) + f"|kf{len(keyframes)}|l{levels}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return tuple(cache[key]["tile"]), cache[key]
    ref = None
    report = {"key": key, "ms_per_step": {}, "identical_image": {}}
    for tw, th in candidates:
        bw = BatchedWindow(_clone(params), keyframes, levels=levels, tiling=tiling_struct(tw, th))
        bw.preprocess()
        bw.bin_sort()
        bw.iterate()
        torch.cuda.synchronize()
        imgs = [t.clone() for t in bw.imgs]
        if ref is None:
            ref = imgs
        same = all(torch.equal(a, b) for a, b in zip(imgs, ref))
        report["identical_image"][f"{tw}x{th}"] = same
        if not same:
            raise RuntimeError(f"tiling {tw}x{th} changed a rendered view")
        # the eager pass above left screen-space gradients behind: clear them
        bw.g2.zero_()
        bw.capture()
        for _ in range(warmup):
            bw.step()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bw.step()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        if bw.status.item() != 0:
            raise RuntimeError(f"tiling {tw}x{th}: device status {bw.status.item():#x}")
        report["ms_per_step"][f"{tw}x{th}"] = statistics.median(times)
        if verbose:
            print(f"autotune window {tw}x{th}: {report['ms_per_step'][f'{tw}x{th}']:.4f} ms/step")
        del bw
    best = min(report["ms_per_step"], key=report["ms_per_step"].get)
    tile = tuple(int(v) for v in best.split("x"))
    report["tile"] = list(tile)
    if cache_path:
        cache[key] = report
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return tile, report
