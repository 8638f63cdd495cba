"""Photorealistic-mapping drivers over the C ABI (Photo-SLAM, arXiv 2311.16728,
Sec. 3.3-3.4).

* `gp_level` / `PlainMapper`: the plain single-view path.  Each iteration
  trains on one keyframe at one Gaussian-pyramid level (Eq. 5); a keyframe
  starts at the coarsest level and moves one level finer every tau_u / levels
  of its uses, reaching level 0 after tau_u uses (the paper gives no switch
  points; this is the schedule's reading).
* `BatchedWindow` (batched.py): every level of every keyframe in one
  iteration.
* `densify_default` / `densify_learned`: new primitives at keypoints
  (Sec. 3.3.1), initialised by the default rule, or by the default rule
  corrected by the learned MLP.
* `Evaluator`: PSNR of the map against level-0 keyframe images.
* `harvest` / `train_initialiser`: (patch, converged parameter) pairs produced
  by a mapping run, and the MLP's training on them.
* `Densifier`: gradient-driven densification and pruning (Sec. 3.3.1) of a
  map kept in a padded store.
"""
from __future__ import annotations

from typing import List, Sequence

import ctypes

import torch

from . import _lib as L
from .learned_init import N3, LearnedInit, default_init
from .raster import (PYRAMID_LEVELS, Adam, AdamConfig, Gaussians, MappingStep, ViewBuffers, _p, camera_at_level,
                     camera_from, ensure_capacity, psnr, pyramid, tiling_struct)

TAU_U = 30  # keyframe uses until level 0 (schedule reading)


def gp_level(use: int, levels: int = PYRAMID_LEVELS, tau_u: int = TAU_U) -> int:
    """Pyramid level of a keyframe at its `use`-th training use (0-based)."""
    per = max(1, tau_u // levels)
    return max(0, levels - 1 - use // per)


class PlainMapper:
    """Single-view mapping with the sequential pyramid schedule: keyframes in
    turn, one (keyframe, level) view per iteration, one CUDA-graph set per
    level sharing the parameters, gradients and Adam state."""

    def __init__(self, params: Gaussians, keyframes: Sequence, levels: int = PYRAMID_LEVELS, tau_u: int = TAU_U,
                 adam_cfg: AdamConfig = AdamConfig(), tiling=None):
        self.params = params
        self.levels, self.tau_u = levels, tau_u
        self.grads = params.zeros_like()
        self.adam = Adam(params, adam_cfg)
        pyrs = [pyramid(gt.contiguous(), levels) for _, gt in keyframes]
        self.steps = []
        for lvl in range(levels):
            views = [(camera_at_level(camera_from(cam), lvl), pyrs[k][lvl]) for k, (cam, _) in enumerate(keyframes)]
            self.steps.append(MappingStep(params, views, tiling, adam=self.adam, grads=self.grads))
        self.nkf = len(keyframes)
        self.uses = [0] * self.nkf
        self.k = 0

    def capture(self):
        for ms in self.steps:
            ms.capture()

    def step(self):
        kf = self.k % self.nkf
        self.steps[gp_level(self.uses[kf], self.levels, self.tau_u)].step_view(kf)
        self.uses[kf] += 1
        self.k += 1

    def status(self) -> int:
        return max(ms.status() for ms in self.steps)


class Evaluator:
    """Mean PSNR (dB) of renders of a map against [(camera, level-0 image)]."""

    def __init__(self, n: int, views: Sequence, tiling=None):
        self.views = [(camera_from(c), gt.contiguous()) for c, gt in views]
        self.vb = ViewBuffers(n, self.views[0][0], tiling or tiling_struct(16, 16), 1024)

    def __call__(self, params: Gaussians) -> float:
        vals = []
        for cam, gt in self.views:
            self.vb.cam = cam
            ensure_capacity(self.vb, params)
            self.vb.forward(params)
            vals.append(psnr(self.vb.img, gt))
        return float(torch.cat(vals).mean().item())


def densify_default(params: Gaussians, keyframes: Sequence, keypoints: Sequence[torch.Tensor],
                    offsets: Sequence[int]):
    """Default initialisation of the new primitives of each keyframe (slots
    offsets[k] .. offsets[k] + len(keypoints[k]) - 1)."""
    for (cam, img), kp, off in zip(keyframes, keypoints, offsets):
        if kp.shape[0]:
            default_init(params, img, kp, cam, off)


def densify_learned(li: LearnedInit, params: Gaussians, keyframes: Sequence, keypoints: Sequence[torch.Tensor],
                    offsets: Sequence[int], levels: int = PYRAMID_LEVELS):
    """The learned initialiser: the default rule first, then the MLP's
    correction of its encoded parameters, predicted from the patches of each
    keyframe's pyramid around its keypoints (tensor cores)."""
    densify_default(params, keyframes, keypoints, offsets)
    dev = params.mean_op.device
    base = torch.zeros(li.mpad, N3, dtype=torch.float32, device=dev)
    for (cam, img), kp, off in zip(keyframes, keypoints, offsets):
        pyr = pyramid(img.contiguous(), levels)
        for s in range(0, kp.shape[0], li.mpad):
            part = kp[s:s + li.mpad]
            M = part.shape[0]
            gids = torch.arange(off + s, off + s + M, dtype=torch.int32, device=dev)
            li.encode_targets(params, gids, part, cam, base)
            li.gather(pyr, part, transpose=False)
            li.forward()
            li.decode(part, cam, params, off + s, base=base)


class Batch:
    """One training batch of the initialiser: x [Mpad, K0] and x^T (BF16),
    target [Mpad, 64] (FP32), M valid rows."""

    def __init__(self, x, xT, target, M):
        self.x, self.xT, self.target, self.M = x, xT, target, M


def harvest(li: LearnedInit, converged: Gaussians, initial: Gaussians, keyframes: Sequence,
            keypoints: Sequence[torch.Tensor], offsets: Sequence[int], levels: int = PYRAMID_LEVELS) -> List[Batch]:
    """(patch, converged parameter) pairs of the primitives a mapping run
    created at keypoints: inputs gathered from each keyframe's pyramid,
    targets = encoded converged parameters minus the encoded initial (default)
    ones (slot offsets[k] + m of keypoint m).  Batches hold at most li.mpad
    rows."""
    out = []
    dev = converged.mean_op.device
    base = torch.zeros(li.mpad, N3, dtype=torch.float32, device=dev)
    for (cam, img), kp, off in zip(keyframes, keypoints, offsets):
        pyr = pyramid(img.contiguous(), levels)
        for s in range(0, kp.shape[0], li.mpad):
            part = kp[s:s + li.mpad]
            M = part.shape[0]
            li.gather(pyr, part, transpose=True)
            gids = torch.arange(off + s, off + s + M, dtype=torch.int32, device=dev)
            target = torch.zeros(li.mpad, N3, dtype=torch.float32, device=dev)
            li.encode_targets(initial, gids, part, cam, base)
            li.encode_targets(converged, gids, part, cam, target, base=base)
            out.append(Batch(li.x.clone(), li.xT.clone(), target, M))
    return out


def train_initialiser(li: LearnedInit, batches: Sequence[Batch], steps: int, seed: int = 0) -> List[float]:
    """`steps` Adam steps of the MLP, each on one batch (seeded random order).
    Returns the loss of every step."""
    g = torch.Generator().manual_seed(seed)
    losses = []
    for _ in range(steps):
        b = batches[int(torch.randint(len(batches), (1,), generator=g))]
        li.train_step(b.target, b.M, x=b.x, xT=b.xT)
        losses.append(li.loss.clone())
    return torch.cat(losses).cpu().tolist() if losses else []


class Densifier:
    """Gradient-driven densification and pruning (Sec. 3.3.1) of a map kept
    in a store with spare capacity: the live Gaussians occupy the first
    `n_live` slots and the rest is inert padding, so that captured
    iterations over the whole store stay valid until the store is full.

    Every mapping iteration adds each seen Gaussian's |dL/d(u, v)| (NDC) to
    `stat` and 1 to `count` (pass them to MappingStep).  `step()` runs
    gsr_densify with seeded standard normals for the split offsets and
    writes the result back into the same store (the captured graphs keep
    their pointers); when the result does not fit it returns a new, larger
    store and the caller re-captures."""

    def __init__(self, params: Gaussians, adam: Adam, n_live: int, grad_thr: float = 2e-4,
                 min_opacity: float = 0.005, split_scale: float = 0.03, shrink: float = 1.6, seed: int = 0,
                 growth: float = 1.25):
        import math
        self.params, self.adam, self.n_live, self.growth = params, adam, n_live, growth
        dev = params.mean_op.device
        self.stat = torch.zeros(params.n, dtype=torch.float32, device=dev)
        self.count = torch.zeros(params.n, dtype=torch.float32, device=dev)
        self.cfg = L.gsr_densify_config(grad_thr, math.log(min_opacity / (1.0 - min_opacity)), math.log(split_scale),
                                        math.log(shrink))
        self.gen = torch.Generator(device=dev).manual_seed(seed)
        self.d_n = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def _run(self, out: Gaussians, om: Gaussians, ov: Gaussians) -> int:
        n = self.n_live
        eps = torch.randn(max(n, 1), 6, generator=self.gen, device=self.params.mean_op.device)
        sz = ctypes.c_size_t()
        L.gsr_densify_workspace_size(n, ctypes.byref(sz))
        ws = torch.empty(sz.value, dtype=torch.uint8, device=eps.device)
        pb = [x.buffers_struct() for x in (self.params, self.adam.m, self.adam.v, out, om, ov)]
        self.status.zero_()
        L.gsr_densify(ctypes.byref(pb[0]), ctypes.byref(pb[1]), ctypes.byref(pb[2]), n, _p(self.stat), _p(self.count),
                      _p(eps), ctypes.byref(self.cfg), ctypes.byref(pb[3]), ctypes.byref(pb[4]), ctypes.byref(pb[5]),
                      out.n, _p(self.d_n), _p(ws), ws.numel(), _p(self.status), None)
        return int(self.d_n.item())

    def step(self):
        """Densify and prune.  Returns (n_live, grown): grown is True when the
        store was replaced by a larger one (self.params / self.adam are then
        new objects and captured iterations must be rebuilt)."""
        cap = self.params.n
        out, om, ov = (Gaussians.zeros(cap, self.params.mean_op.device, self.params.sh_degree) for _ in range(3))
        n_out = self._run(out, om, ov)
        grown = n_out > cap
        if grown:
            cap = int(n_out * self.growth) + 1024
            out, om, ov = (Gaussians.zeros(cap, self.params.mean_op.device, self.params.sh_degree) for _ in range(3))
            n_out = self._run(out, om, ov)
            adam = Adam(out, self.adam.cfg)
            adam.m, adam.v = om, ov
            adam.step_count.copy_(self.adam.step_count)
            self.params, self.adam = out, adam
            dev = out.mean_op.device
            self.stat = torch.zeros(cap, dtype=torch.float32, device=dev)
            self.count = torch.zeros(cap, dtype=torch.float32, device=dev)
        else:
            for dst, src in zip([t for x in (self.params, self.adam.m, self.adam.v) for t in x.tensors()],
                                [t for x in (out, om, ov) for t in x.tensors()]):
                dst.copy_(src)
            self.stat.zero_()
            self.count.zero_()
        self.n_live = n_out
        return n_out, grown
