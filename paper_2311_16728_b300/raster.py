"""Torch-facing glue over the libgsr C ABI: buffers, the autograd Function and
the captured mapping iteration of Photo-SLAM's photorealistic mapping
(arXiv 2311.16728, Sec. 3.3 Eq. 3-4, Sec. 3.4 Eq. 5).

PyTorch only allocates device memory, provides streams and CUDA graphs, and
carries autograd bookkeeping; every arithmetic step runs in libgsr's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

LAMBDA_DSSIM = 0.2  # Eq. 4 weight, Sec. 4.1
PYRAMID_LEVELS = 3  # n = 2 -> three levels, Sec. 4.1


def _p(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- parameters
@dataclass
class Gaussians:
    """SoA parameter store on the device (see include/gsr.h for the layout)."""
    mean_op: torch.Tensor   # (N, 4)
    quat: torch.Tensor      # (N, 4)
    logscale: torch.Tensor  # (N, 4)
    sh: torch.Tensor        # (12, N, 4)
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return self.mean_op.shape[0]

    @staticmethod
    def from_arrays(mean_op, quat, logscale, sh, sh_degree: int = 3, device="cuda") -> "Gaussians":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device).contiguous()
        return Gaussians(f(mean_op), f(quat), f(logscale), f(sh), sh_degree)

    @staticmethod
    def zeros(n: int, device="cuda", sh_degree: int = 3) -> "Gaussians":
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        return Gaussians(z(n, 4), z(n, 4), z(n, 4), z(12, n, 4), sh_degree)

    def zeros_like(self) -> "Gaussians":
        return Gaussians(torch.zeros_like(self.mean_op), torch.zeros_like(self.quat),
                         torch.zeros_like(self.logscale), torch.zeros_like(self.sh), self.sh_degree)

    def tensors(self):
        return (self.mean_op, self.quat, self.logscale, self.sh)

    def gaussians_struct(self) -> L.gsr_gaussians:
        return L.gsr_gaussians(self.mean_op.data_ptr(), self.quat.data_ptr(), self.logscale.data_ptr(),
                               self.sh.data_ptr(), self.n, self.sh_degree)

    def buffers_struct(self) -> L.gsr_param_buffers:
        return L.gsr_param_buffers(self.mean_op.data_ptr(), self.quat.data_ptr(), self.logscale.data_ptr(),
                                   self.sh.data_ptr())


def spatial_order(params: Gaussians, lo, hi) -> torch.Tensor:
    """Permutation (n int32, device) that sorts the Gaussians by the Morton
    code of their means in the box [lo, hi] (gsr_spatial_order)."""
    n = params.n
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=params.mean_op.device)
    sz = ctypes.c_size_t()
    L.gsr_spatial_order_workspace_size(n, ctypes.byref(sz))
    ws = torch.empty(sz.value, dtype=torch.uint8, device=params.mean_op.device)
    gs = params.gaussians_struct()
    lo3, hi3 = (ctypes.c_float * 3)(*[float(v) for v in lo]), (ctypes.c_float * 3)(*[float(v) for v in hi])
    L.gsr_spatial_order(ctypes.byref(gs), lo3, hi3, _p(perm), _p(ws), ws.numel(), _stream(None))
    return perm[:n]


def permuted(x: Gaussians, perm: torch.Tensor) -> Gaussians:
    """A new store with entry i = x's entry perm[i] (gsr_permute)."""
    out = x.zeros_like()
    src, dst = x.buffers_struct(), out.buffers_struct()
    L.gsr_permute(ctypes.byref(src), ctypes.byref(dst), _p(perm), x.n, _stream(None))
    return out


def camera_struct(R, t, fx, fy, cx, cy, width, height) -> L.gsr_camera:
    c = L.gsr_camera()
    c.R[:] = [float(v) for v in np.asarray(R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(t, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.width, c.height = int(width), int(height)
    return c


def camera_from(obj) -> L.gsr_camera:
    """Any object with R, t, fx, fy, cx, cy, width, height attributes."""
    if isinstance(obj, L.gsr_camera):
        return obj
    return camera_struct(obj.R, obj.t, obj.fx, obj.fy, obj.cx, obj.cy, obj.width, obj.height)


def camera_at_level(cam: L.gsr_camera, level: int) -> L.gsr_camera:
    out = L.gsr_camera()
    L.gsr_camera_at_level(ctypes.byref(cam), int(level), ctypes.byref(out))
    return out


def tiling_struct(tile_w: int = 16, tile_h: int = 16, batch_depth: int = 0, bwd_threads: int = 0) -> L.gsr_tiling:
    """Tile shape and the blend kernels' staging batch depth and backward
    threads per tile (0 = the defaults); none of them changes the image."""
    return L.gsr_tiling(int(tile_w), int(tile_h), int(batch_depth), int(bwd_threads))


def n_tiles(cam: L.gsr_camera, tiling: L.gsr_tiling) -> int:
    return ((cam.width + tiling.tile_w - 1) // tiling.tile_w) * ((cam.height + tiling.tile_h - 1) // tiling.tile_h)


# ---------------------------------------------------------------- one view
class ViewBuffers:
    """Every device buffer one view of the hot path needs, allocated once.

    `pair_capacity` bounds the (Gaussian, tile) pairs; overflow is reported
    through the status word, never written out of bounds.
    """

    def __init__(self, n: int, cam: L.gsr_camera, tiling: L.gsr_tiling, pair_capacity: int, device="cuda"):
        self.n, self.cam, self.tiling = n, cam, tiling
        self.device = device
        f32 = dict(dtype=torch.float32, device=device)
        m = max(n, 1)  # keep every buffer a real allocation, also for an empty map
        self.xy_conic = torch.empty(m, 4, **f32)
        self.c_op_box = torch.empty(m, 4, **f32)
        self.rgb_depth = torch.empty(m, 4, **f32)
        self.ntiles = torch.zeros(m, dtype=torch.int32, device=device)
        self.uv_lo = torch.zeros(m, 2, **f32)
        self.tiles = n_tiles(cam, tiling)
        self.ranges = torch.zeros(self.tiles, 2, dtype=torch.int32, device=device)
        # tiles by decreasing pair count (binning writes it, the blends read it)
        self.tile_order = torch.arange(self.tiles, dtype=torch.int32, device=device)
        # per-tile depth of list the backward walks (the forward writes it; the backward's order)
        self.tile_work = torch.zeros(self.tiles, dtype=torch.int32, device=device)
        self.num_pairs = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        H, W = cam.height, cam.width
        self.img = torch.empty(3, H, W, **f32)
        self.T_final = torch.empty(H, W, **f32)
        self.n_contrib = torch.empty(H, W, dtype=torch.int32, device=device)
        self.dimg = torch.empty(3, H, W, **f32)
        self.loss = torch.zeros(1, **f32)
        self.g2 = torch.zeros(3, m, 4, **f32)
        sz = ctypes.c_size_t()
        L.gsr_loss_workspace_size(3, H, W, ctypes.byref(sz))
        self.loss_ws = torch.empty(max(int(sz.value), 1), dtype=torch.uint8, device=device)
        self.set_pair_capacity(pair_capacity)

    def set_pair_capacity(self, cap: int):
        self.pair_capacity = int(cap)
        self.keys = torch.empty(max(self.pair_capacity, 1), dtype=torch.int64, device=self.device)
        self.vals = torch.empty(max(self.pair_capacity, 1), dtype=torch.int32, device=self.device)
        sz = ctypes.c_size_t()
        L.gsr_bin_sort_workspace_size(self.n, self.pair_capacity, ctypes.byref(self.cam), ctypes.byref(self.tiling),
                                      ctypes.byref(sz))
        self.sort_ws = torch.empty(max(int(sz.value), 1), dtype=torch.uint8, device=self.device)

    def proj_struct(self) -> L.gsr_proj:
        return L.gsr_proj(self.xy_conic.data_ptr(), self.c_op_box.data_ptr(), self.rgb_depth.data_ptr(),
                          self.ntiles.data_ptr(), self.uv_lo.data_ptr(), self.tile_order.data_ptr(),
                          self.tile_work.data_ptr())

    def grad2d_struct(self) -> L.gsr_grad2d:
        return L.gsr_grad2d(self.g2[0].data_ptr(), self.g2[1].data_ptr(), self.g2[2].data_ptr())

    # -- the calls, in hot-path order ------------------------------------
    def preprocess(self, g: Gaussians, stream=None):
        gs, proj = g.gaussians_struct(), self.proj_struct()
        L.gsr_preprocess(ctypes.byref(gs), ctypes.byref(self.cam), ctypes.byref(self.tiling), ctypes.byref(proj),
                         _p(self.status), _stream(stream))

    def bin_sort(self, stream=None):
        proj = self.proj_struct()
        L.gsr_bin_sort(ctypes.byref(proj), self.n, ctypes.byref(self.cam), ctypes.byref(self.tiling), _p(self.keys),
                       _p(self.vals), self.pair_capacity, _p(self.ranges), _p(self.num_pairs), _p(self.sort_ws),
                       self.sort_ws.numel(), _p(self.status), _stream(stream))

    def render_fwd(self, bg: Sequence[float] = (0.0, 0.0, 0.0), stream=None, n_blended=None):
        proj = self.proj_struct()
        bga = (ctypes.c_float * 3)(*bg)
        L.gsr_render_fwd(ctypes.byref(proj), _p(self.vals), _p(self.ranges), ctypes.byref(self.cam),
                         ctypes.byref(self.tiling), bga, _p(self.img), _p(self.T_final), _p(self.n_contrib),
                         _p(n_blended), _stream(stream))

    def loss_fwd_bwd(self, gt: torch.Tensor, lam: float = LAMBDA_DSSIM, stream=None):
        """Eq. 4 against gt: an RGB target (3 x H x W), or a grayscale one
        (1 x H x W), then on the render's luminance."""
        H, W = self.cam.height, self.cam.width
        if gt.shape[0] == 1:
            sz = ctypes.c_size_t()
            L.gsr_loss_luma_workspace_size(H, W, ctypes.byref(sz))
            if self.loss_ws.numel() < sz.value:
                self.loss_ws = torch.empty(int(sz.value), dtype=torch.uint8, device=self.img.device)
            L.gsr_loss_luma_fwd_bwd(_p(self.img), _p(gt), H, W, float(lam), _p(self.loss), _p(self.dimg),
                                    _p(self.loss_ws), self.loss_ws.numel(), _stream(stream))
            return
        L.gsr_loss_fwd_bwd(_p(self.img), _p(gt), 3, H, W, float(lam), _p(self.loss), _p(self.dimg),
                           _p(self.loss_ws), self.loss_ws.numel(), _stream(stream))

    def render_bwd(self, g: Gaussians, grads: Gaussians, dimg: Optional[torch.Tensor] = None,
                   bg: Sequence[float] = (0.0, 0.0, 0.0), densify_stat=None, densify_count=None, stream=None):
        gs, proj, g2, gb = g.gaussians_struct(), self.proj_struct(), self.grad2d_struct(), grads.buffers_struct()
        bga = (ctypes.c_float * 3)(*bg)
        d = self.dimg if dimg is None else dimg
        L.gsr_render_bwd(ctypes.byref(gs), ctypes.byref(proj), _p(self.vals), _p(self.ranges), ctypes.byref(self.cam),
                         ctypes.byref(self.tiling), bga, _p(self.T_final), _p(self.n_contrib), _p(d),
                         ctypes.byref(g2), ctypes.byref(gb), _p(densify_stat), _p(densify_count), _stream(stream))

    def blend_bwd(self, dimg: Optional[torch.Tensor] = None, bg: Sequence[float] = (0.0, 0.0, 0.0), stream=None):
        proj, g2 = self.proj_struct(), self.grad2d_struct()
        bga = (ctypes.c_float * 3)(*bg)
        d = self.dimg if dimg is None else dimg
        L.gsr_blend_bwd(ctypes.byref(proj), self.n, _p(self.vals), _p(self.ranges), ctypes.byref(self.cam),
                        ctypes.byref(self.tiling), bga, _p(self.T_final), _p(self.n_contrib), _p(d), ctypes.byref(g2),
                        _stream(stream))

    def preprocess_bwd(self, g: Gaussians, grads: Gaussians, densify_stat=None, densify_count=None, stream=None,
                       store: bool = False):
        """Chain rule into `grads`: += (default), or = for the visible
        Gaussians when the caller knows their gradients are zero."""
        gs, proj, g2, gb = g.gaussians_struct(), self.proj_struct(), self.grad2d_struct(), grads.buffers_struct()
        fn = L.gsr_preprocess_bwd_store if store else L.gsr_preprocess_bwd
        fn(ctypes.byref(gs), ctypes.byref(proj), ctypes.byref(self.cam), ctypes.byref(self.tiling), ctypes.byref(g2),
           ctypes.byref(gb), _p(densify_stat), _p(densify_count), _stream(stream))

    def pose_bwd(self, g: Gaussians, d_pose: torch.Tensor, stream=None):
        """Camera pose gradient (+= into d_pose, 15 floats: dL/dR, dL/dt,
        dL/dphi) from the screen-space gradients blend_bwd left in g2."""
        assert d_pose.dtype == torch.float32 and d_pose.numel() >= 15
        gs, proj, g2 = g.gaussians_struct(), self.proj_struct(), self.grad2d_struct()
        L.gsr_pose_bwd(ctypes.byref(gs), ctypes.byref(proj), ctypes.byref(self.cam), ctypes.byref(self.tiling),
                       ctypes.byref(g2), _p(d_pose), _stream(stream))

    def forward(self, g: Gaussians, bg=(0.0, 0.0, 0.0), stream=None):
        self.preprocess(g, stream)
        self.bin_sort(stream)
        self.render_fwd(bg, stream)

    def read_status(self) -> int:
        torch.cuda.current_stream().synchronize()
        return int(self.status.item())

    def pairs_needed(self) -> int:
        return int(self.num_pairs.item())


def ensure_capacity(vb: ViewBuffers, g: Gaussians, bg=(0.0, 0.0, 0.0), margin: float = 1.3) -> bool:
    """Run the binning once; grow the pair capacity if it overflowed.  Syncs."""
    vb.status.zero_()
    vb.preprocess(g)
    vb.bin_sort()
    need = vb.pairs_needed()
    grown = need > vb.pair_capacity
    if grown:
        vb.set_pair_capacity(int(need * margin) + 1024)
    vb.status.zero_()
    return grown


# ---------------------------------------------------------------- autograd
class RasterizeGaussians(torch.autograd.Function):
    """img = render(mean_op, quat, logscale, sh; camera).

    Forward runs preprocess -> bin/sort -> blend; backward replays the blend
    from the saved T_final / n_contrib (no per-pixel lists are stored) and
    chains to all parameters.  One forward per ViewBuffers may be in flight
    (its buffers hold the saved state).
    """

    @staticmethod
    def forward(ctx, mean_op, quat, logscale, sh, vb: ViewBuffers, sh_degree: int, bg):
        g = Gaussians(mean_op.detach().contiguous(), quat.detach().contiguous(), logscale.detach().contiguous(),
                      sh.detach().contiguous(), sh_degree)
        ensure_capacity(vb, g, bg)
        vb.forward(g, bg)
        ctx.vb, ctx.g, ctx.bg = vb, g, bg
        return vb.img.clone()

    @staticmethod
    def backward(ctx, dimg):
        vb, g = ctx.vb, ctx.g
        grads = g.zeros_like()
        vb.render_bwd(g, grads, dimg=dimg.contiguous(), bg=ctx.bg)
        return grads.mean_op, grads.quat, grads.logscale, grads.sh, None, None, None


def rasterize(g_mean_op, g_quat, g_logscale, g_sh, vb: ViewBuffers, sh_degree: int = 3, bg=(0.0, 0.0, 0.0)):
    return RasterizeGaussians.apply(g_mean_op, g_quat, g_logscale, g_sh, vb, sh_degree, tuple(bg))


# ---------------------------------------------------------------- optimiser
@dataclass
class AdamConfig:
    lr_mean: float = 1.6e-4
    lr_opacity: float = 5e-2
    lr_quat: float = 1e-3
    lr_scale: float = 5e-3
    lr_sh: float = 2.5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15

    def struct(self) -> L.gsr_adam_config:
        return L.gsr_adam_config(self.lr_mean, self.lr_opacity, self.lr_quat, self.lr_scale, self.lr_sh,
                                 self.beta1, self.beta2, self.eps)


class Adam:
    def __init__(self, params: Gaussians, cfg: AdamConfig = AdamConfig()):
        self.params, self.cfg = params, cfg
        self.m, self.v = params.zeros_like(), params.zeros_like()
        self.step_count = torch.zeros(1, dtype=torch.int32, device=params.mean_op.device)
        self._cfg = cfg.struct()

    def step(self, grads: Gaussians, stream=None, touched: Optional[torch.Tensor] = None):
        """One step; `touched` (n int32 flags, optional): Gaussians whose flag is
        0 are known to have a zero gradient, which is then not read."""
        p, g, m, v = (x.buffers_struct() for x in (self.params, grads, self.m, self.v))
        if touched is None:
            L.gsr_adam_step(ctypes.byref(p), ctypes.byref(g), ctypes.byref(m), ctypes.byref(v), self.params.n,
                            ctypes.byref(self._cfg), _p(self.step_count), _stream(stream))
        else:
            L.gsr_adam_step_touched(ctypes.byref(p), ctypes.byref(g), ctypes.byref(m), ctypes.byref(v),
                                    self.params.n, ctypes.byref(self._cfg), _p(touched), _p(self.step_count),
                                    _stream(stream))


def pyramid(img: torch.Tensor, levels: int = PYRAMID_LEVELS, stream=None):
    """[GP^0(img), ..., GP^{levels-1}(img)] (Eq. 5)."""
    out = [img.contiguous()]
    for _ in range(levels - 1):
        C, H, W = out[-1].shape
        nxt = torch.empty(C, (H + 1) // 2, (W + 1) // 2, dtype=torch.float32, device=img.device)
        L.gsr_pyramid_down(_p(out[-1]), C, H, W, _p(nxt), _stream(stream))
        out.append(nxt)
    return out


def psnr(img: torch.Tensor, gt: torch.Tensor, stream=None) -> torch.Tensor:
    sz = ctypes.c_size_t()
    L.gsr_psnr_workspace_size(img.numel(), ctypes.byref(sz))
    ws = torch.empty(int(sz.value), dtype=torch.uint8, device=img.device)
    out = torch.zeros(1, dtype=torch.float32, device=img.device)
    L.gsr_psnr(_p(img.contiguous()), _p(gt.contiguous()), img.numel(), _p(out), _p(ws), ws.numel(), _stream(stream))
    return out


# ---------------------------------------------------------------- mapping step
STAGES = ("preprocess", "bin_sort", "render_fwd", "loss", "blend_bwd", "preprocess_bwd", "adam")


class MappingStep:
    """One photorealistic-mapping iteration over one view (Sec. 3.3):
    preprocess -> bin/sort -> render -> Eq. 4 loss + dL/dI -> backward -> Adam.

    `views` is a list of (camera, gt image) pairs sharing one resolution; each
    call to `step()` trains on the next view.  `capture()` records every view's
    iteration as one CUDA graph (the camera struct is baked into each launch),
    and also as one graph per stage, so that CUDA events between stages can
    time them live (`step(events=...)` replays those).
    """

    def __init__(self, params: Gaussians, views, tiling: L.gsr_tiling = None, adam_cfg: AdamConfig = AdamConfig(),
                 lam: float = LAMBDA_DSSIM, pair_capacity: Optional[int] = None, margin: float = 1.5,
                 adam: Optional[Adam] = None, grads: Optional[Gaussians] = None,
                 densify_stat: Optional[torch.Tensor] = None, densify_count: Optional[torch.Tensor] = None):
        """`adam` and `grads` may be shared with other steps over the same
        parameters (e.g. one step per pyramid level); with densify_stat /
        densify_count (n floats each) every iteration accumulates the
        densification statistic of the Gaussians it sees."""
        self.params = params
        self.densify_stat, self.densify_count = densify_stat, densify_count
        self.tiling = tiling or tiling_struct(16, 16)
        self.views = [(camera_from(c), gt.contiguous()) for c, gt in views]
        self.lam = lam
        self.grads = grads if grads is not None else params.zeros_like()
        self.adam = adam if adam is not None else Adam(params, adam_cfg)
        cam0 = self.views[0][0]
        self.vb = ViewBuffers(params.n, cam0, self.tiling, pair_capacity or 1024)
        if pair_capacity is None:
            need = 0
            for cam, _ in self.views:
                self.vb.cam = cam
                self.vb.status.zero_()
                self.vb.preprocess(params)
                self.vb.bin_sort()
                need = max(need, self.vb.pairs_needed())
            self.vb.set_pair_capacity(int(need * margin) + 4096)
        self.vb.status.zero_()  # the sizing passes may have flagged overflow
        self.vb.cam = cam0
        self.graphs = None
        self.whole = None
        self.k = 0

    def _stage(self, idx: int, name: str, stream=None):
        cam, gt = self.views[idx]
        vb = self.vb
        vb.cam = cam
        if name == "preprocess":
            vb.preprocess(self.params, stream)
        elif name == "bin_sort":
            vb.bin_sort(stream)
        elif name == "render_fwd":
            vb.render_fwd(stream=stream)
        elif name == "loss":
            vb.loss_fwd_bwd(gt, self.lam, stream)
        elif name == "blend_bwd":
            vb.blend_bwd(stream=stream)
        elif name == "preprocess_bwd":
            # the gradients are zero here (Adam zeroes what it reads), so the
            # chain rule stores them instead of adding
            vb.preprocess_bwd(self.params, self.grads, self.densify_stat, self.densify_count, stream=stream,
                              store=True)
        elif name == "adam":
            # the one-view backward writes gradients exactly where ntiles > 0
            self.adam.step(self.grads, stream, touched=vb.ntiles if self.params.n else None)

    def _run(self, idx: int, stream=None):
        for name in STAGES:
            self._stage(idx, name, stream)

    def _snapshot(self):
        return [t.clone() for x in (self.params, self.adam.m, self.adam.v) for t in x.tensors()], \
            self.adam.step_count.clone()

    def _restore(self, snap):
        saved, step0 = snap
        for dst, src in zip([t for x in (self.params, self.adam.m, self.adam.v) for t in x.tensors()], saved):
            dst.copy_(src)
        self.adam.step_count.copy_(step0)

    def capture(self):
        """Capture one CUDA graph per view (the whole iteration) and one per
        (view, stage)."""
        # one eager iteration loads every kernel before capture; its effect on
        # the parameters, moments and step counter is undone afterwards
        snap = self._snapshot()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._run(0, s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self._restore(snap)
        torch.cuda.synchronize()
        self.graphs = []
        for i in range(len(self.views)):
            per = []
            for name in STAGES:
                gph = torch.cuda.CUDAGraph(keep_graph=True)  # kept for kernel-node counting
                with torch.cuda.graph(gph):
                    self._stage(i, name, torch.cuda.current_stream())
                gph.instantiate()
                per.append(gph)
            self.graphs.append(per)
        self.whole = []
        for i in range(len(self.views)):
            gph = torch.cuda.CUDAGraph(keep_graph=True)
            with torch.cuda.graph(gph):
                self._run(i, torch.cuda.current_stream())
            gph.instantiate()
            self.whole.append(gph)
        self.vb.cam = self.views[0][0]

    def step(self, events=None):
        """One iteration on the next view.  `events` (optional) is a list of
        len(STAGES) + 1 CUDA events recorded before the first and after every
        stage on the current stream."""
        self.step_view(self.k % len(self.views), events)

    def step_view(self, i: int, events=None):
        """One iteration on view i: one graph replay, or (with events) one
        replay per stage with the events between them."""
        if events is None and self.whole is not None:
            self.whole[i].replay()
            self.k += 1
            return
        if events is not None:
            events[0].record()
        for si, name in enumerate(STAGES):
            if self.graphs is not None:
                self.graphs[i][si].replay()
            else:
                self._stage(i, name)
            if events is not None:
                events[si + 1].record()
        self.k += 1

    def status(self) -> int:
        return self.vb.read_status()
