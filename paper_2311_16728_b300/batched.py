"""Batched Gaussian-pyramid window (Sec. 3.4, Eq. 5) as one captured iteration.

All (keyframe, level) views of a window are optimised together: one batched
projection, one binning, ONE persistent launch for the forward blend, the
Eq. 4 loss and its gradient, and the backward blend of every view, then the
summed chain rule and Adam -- captured once as a CUDA graph and replayed.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib as L
from .raster import (LAMBDA_DSSIM, PYRAMID_LEVELS, Adam, AdamConfig, Gaussians, _p, _stream, camera_at_level,
                     camera_from, n_tiles, pyramid, tiling_struct)


class BatchedWindow:
    """views: every (keyframe, level) of `keyframes` = [(camera, level-0 gt)],
    coarsest level first; `views[v]` = (camera, gt, level, keyframe index)."""

    def __init__(self, params: Gaussians, keyframes: Sequence, levels: int = PYRAMID_LEVELS,
                 weights: Optional[Sequence[float]] = None, adam_cfg: AdamConfig = AdamConfig(),
                 lam: float = LAMBDA_DSSIM, pair_capacity: Optional[int] = None, margin: float = 1.5,
                 tiling: Optional[L.gsr_tiling] = None):
        self.params = params
        self.tiling = tiling or tiling_struct(16, 16)
        self.lam = lam
        dev = params.mean_op.device
        pyr = [pyramid(gt.contiguous(), levels) for _, gt in keyframes]
        views = []
        # coarsest level first: its tiles carry the longest lists, and taking
        # the longest work items first keeps the tail of each phase short
        for l in reversed(range(levels)):
            for k, (cam, _) in enumerate(keyframes):
                views.append((camera_at_level(camera_from(cam), l), pyr[k][l], l, k))
        self.views = views
        V = len(views)
        assert V <= 64, "at most 64 views per window"
        self.V = V
        self.cams = (L.gsr_camera * V)(*[v[0] for v in views])
        n = params.n
        self.n = n
        f32 = dict(dtype=torch.float32, device=dev)
        m = max(n, 1) * V
        self.xy_conic = torch.empty(m, 4, **f32)
        self.c_op_box = torch.empty(m, 4, **f32)
        self.rgb_depth = torch.empty(m, 4, **f32)
        self.ntiles = torch.zeros(m, dtype=torch.int32, device=dev)
        self.uv_lo = torch.zeros(m, 2, **f32)
        # the visible records gathered densely by the binning (the pairs'
        # values index these; rec_to_c maps a record to its position), so the
        # persistent launch and the chain rule touch arrays that stay in L2
        self.cxy = torch.empty(m, 4, **f32)
        self.ccb = torch.empty(m, 4, **f32)
        self.crd = torch.empty(m, 4, **f32)
        self.cuv = torch.zeros(m, 2, **f32)
        self.rec_to_c = torch.zeros(m, dtype=torch.int32, device=dev)
        self.tiles = sum(n_tiles(v[0], self.tiling) for v in views)
        self.ranges = torch.zeros(self.tiles, 2, dtype=torch.int32, device=dev)
        # tiles of all views by decreasing pair count (binning writes it, the persistent launch reads it)
        self.tile_order = torch.arange(self.tiles, dtype=torch.int32, device=dev)
        self.num_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.imgs = [torch.empty(3, v[0].height, v[0].width, **f32) for v in views]
        self.T = [torch.empty(v[0].height, v[0].width, **f32) for v in views]
        self.nc = [torch.empty(v[0].height, v[0].width, dtype=torch.int32, device=dev) for v in views]
        self.dimg = [torch.empty(3, v[0].height, v[0].width, **f32) for v in views]
        self.gts = [v[1].contiguous() for v in views]
        self.losses = torch.zeros(V, **f32)
        self.g2 = torch.zeros(3, m, 4, **f32)  # zero on entry; the chain step leaves it zero
        self.grads = params.zeros_like()
        self.touched = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)  # Gaussians some view saw
        self.adam = Adam(params, adam_cfg)
        self.weights = (ctypes.c_float * V)(*(weights if weights is not None else [1.0] * V))
        ptrs = lambda ts: (ctypes.c_void_p * V)(*[t.data_ptr() for t in ts])
        self.p_img, self.p_T, self.p_nc = ptrs(self.imgs), ptrs(self.T), ptrs(self.nc)
        self.p_gt, self.p_dimg = ptrs(self.gts), ptrs(self.dimg)
        sz = ctypes.c_size_t()
        L.gsr_batched_iterate_workspace_size(self.cams, V, ctypes.byref(sz))
        self.iter_ws = torch.empty(sz.value, dtype=torch.uint8, device=dev)
        self.bg = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
        self._set_capacity(pair_capacity or 1 << 20)
        if pair_capacity is None:
            self.preprocess()
            self.bin_sort()
            need = int(self.num_pairs.item())
            self._set_capacity(int(need * margin) + 4096)
            self.status.zero_()
        self.graph = None
        self.stage_graphs = None

    def set_targets(self, gts):
        """Points the window at another set of target images (one per view,
        the same shapes); capture() afterwards bakes them into a new graph.
        Two graphs over two target sets let one set be refilled while the
        other is in use."""
        assert len(gts) == self.V
        self.gts = [g.contiguous() for g in gts]
        self.p_gt = (ctypes.c_void_p * self.V)(*[t.data_ptr() for t in self.gts])

    def _set_capacity(self, cap: int):
        dev = self.params.mean_op.device
        self.cap = int(cap)
        self.keys = torch.empty(self.cap, dtype=torch.int64, device=dev)
        self.vals = torch.empty(self.cap, dtype=torch.int32, device=dev)
        sz = ctypes.c_size_t()
        L.gsr_bin_sort_workspace_size(self.n * self.V, self.cap, None, ctypes.byref(self.tiling), ctypes.byref(sz))
        self.sort_ws = torch.empty(sz.value, dtype=torch.uint8, device=dev)

    def proj(self) -> L.gsr_proj:
        return L.gsr_proj(self.xy_conic.data_ptr(), self.c_op_box.data_ptr(), self.rgb_depth.data_ptr(),
                          self.ntiles.data_ptr(), self.uv_lo.data_ptr(), self.tile_order.data_ptr())

    def compact(self) -> L.gsr_proj:
        return L.gsr_proj(self.cxy.data_ptr(), self.ccb.data_ptr(), self.crd.data_ptr(), self.rec_to_c.data_ptr(),
                          self.cuv.data_ptr(), self.tile_order.data_ptr())

    def grad2d(self) -> L.gsr_grad2d:
        return L.gsr_grad2d(self.g2[0].data_ptr(), self.g2[1].data_ptr(), self.g2[2].data_ptr())

    # -- the calls of one iteration ------------------------------------------
    def preprocess(self, stream=None):
        gs, pr = self.params.gaussians_struct(), self.proj()
        L.gsr_batched_preprocess(ctypes.byref(gs), self.cams, self.V, ctypes.byref(self.tiling), ctypes.byref(pr),
                                 _stream(stream))

    def bin_sort(self, stream=None):
        pr, cp = self.proj(), self.compact()
        L.gsr_batched_bin_sort(ctypes.byref(pr), self.n, self.cams, self.V, ctypes.byref(self.tiling), _p(self.keys),
                               _p(self.vals), self.cap, _p(self.ranges), _p(self.num_pairs), ctypes.byref(cp),
                               _p(self.sort_ws), self.sort_ws.numel(), _p(self.status), _stream(stream))

    def iterate(self, stream=None):
        pr, g2 = self.compact(), self.grad2d()
        L.gsr_batched_iterate(ctypes.byref(pr), _p(self.vals), _p(self.ranges), self.cams, self.V,
                              ctypes.byref(self.tiling), self.bg, self.p_img, self.p_T, self.p_nc, self.p_gt,
                              self.p_dimg, self.weights, self.lam, _p(self.losses), ctypes.byref(g2), _p(self.iter_ws),
                              self.iter_ws.numel(), _p(self.status), _stream(stream))

    def phase_ms(self):
        """Phase split of the last persistent launch (ms): forward blend,
        SSIM moments, dL/dI, and (entry to barrier 3) for the backward's start
        (the backward's end is the launch's end, timed by the caller)."""
        tail = self.iter_ws[self.iter_ws.numel() - 256 + 64:self.iter_ws.numel() - 256 + 96]
        t = tail.view(torch.int64).cpu().tolist()
        return {"fwd_blend": (t[1] - t[0]) * 1e-6, "ssim_moments": (t[2] - t[1]) * 1e-6,
                "ssim_grad": (t[3] - t[2]) * 1e-6, "entry_to_bwd": (t[3] - t[0]) * 1e-6}

    def chain(self, stream=None):
        gs, pr, cp = self.params.gaussians_struct(), self.proj(), self.compact()
        g2, gb = self.grad2d(), self.grads.buffers_struct()
        L.gsr_batched_preprocess_bwd(ctypes.byref(gs), ctypes.byref(pr), ctypes.byref(cp), self.cams, self.V, ctypes.byref(self.tiling),
                                     ctypes.byref(g2), ctypes.byref(gb), _p(self.touched), _stream(stream))

    STAGES = ("preprocess", "bin_sort", "iterate", "chain", "adam")

    def _stage(self, name: str, stream=None):
        if name == "adam":
            self.adam.step(self.grads, stream, touched=self.touched)
        else:
            getattr(self, name)(stream)

    def _run(self, stream=None):
        for name in self.STAGES:
            self._stage(name, stream)

    def _snapshot(self):
        return [t.clone() for x in (self.params, self.adam.m, self.adam.v) for t in x.tensors()], \
            self.adam.step_count.clone()

    def _restore(self, snap):
        saved, step0 = snap
        for dst, src in zip([t for x in (self.params, self.adam.m, self.adam.v) for t in x.tensors()], saved):
            dst.copy_(src)
        self.adam.step_count.copy_(step0)

    def capture(self, per_stage: bool = False):
        """Captures the whole iteration as ONE CUDA graph (per_stage=False) or
        one graph per stage, so that events between stages time them live.
        One eager warm-up iteration loads the kernels first; its effect on the
        parameters, moments and step counter is undone."""
        snap = self._snapshot()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._run(s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self._restore(snap)
        torch.cuda.synchronize()
        if per_stage:
            self.graph = None
            self.stage_graphs = []
            for name in self.STAGES:
                gph = torch.cuda.CUDAGraph(keep_graph=True)
                with torch.cuda.graph(gph):
                    self._stage(name, torch.cuda.current_stream())
                gph.instantiate()
                self.stage_graphs.append(gph)
        else:
            self.stage_graphs = None
            self.graph = torch.cuda.CUDAGraph(keep_graph=True)  # kept for kernel-node counting
            with torch.cuda.graph(self.graph):
                self._run(torch.cuda.current_stream())
            self.graph.instantiate()

    def graphs(self):
        return [self.graph] if self.graph is not None else list(self.stage_graphs or [])

    def step(self, events=None):
        """One iteration over the whole window.  `events` (per-stage capture
        only): len(STAGES) + 1 CUDA events recorded around the stages."""
        if getattr(self, "stage_graphs", None):
            if events is not None:
                events[0].record()
            for i, gph in enumerate(self.stage_graphs):
                gph.replay()
                if events is not None:
                    events[i + 1].record()
        elif self.graph is not None:
            self.graph.replay()
        else:
            self._run()
