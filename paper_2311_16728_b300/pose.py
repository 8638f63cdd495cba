"""Photometric camera pose refinement against a fixed map: the camera pose
gradient of the Eq. 4 loss through the Eq. 3 render (gsr_pose_bwd, on the
GPU) and Adam steps on the pose's se(3) tangent (six numbers, on the host).

The pose is world->camera (R, t); a step applies the left perturbation
R <- exp([phi]x) R, t <- exp([phi]x) t + rho, whose gradient is
(dL/drho, dL/dphi) = (dL/dt, d_pose[12:15]).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from .raster import LAMBDA_DSSIM, Gaussians, ViewBuffers, camera_from, camera_struct, ensure_capacity, tiling_struct


def so3_exp(phi) -> np.ndarray:
    """Rotation matrix of the axis-angle vector phi (Rodrigues' formula)."""
    phi = np.asarray(phi, np.float64)
    a = float(np.linalg.norm(phi))
    K = np.array([[0.0, -phi[2], phi[1]], [phi[2], 0.0, -phi[0]], [-phi[1], phi[0], 0.0]])
    if a < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + np.sin(a) / a * K + (1.0 - np.cos(a)) / (a * a) * (K @ K)


class PoseRefiner:
    """Refines the pose of one frame (gt: 3 x H x W, or 1 x H x W grayscale
    for the luminance loss) against the map `params`, starting from `cam`."""

    def __init__(self, params: Gaussians, cam, gt: torch.Tensor, lam: float = LAMBDA_DSSIM, tiling=None,
                 lr_rot: float = 2e-3, lr_trans: float = 4e-3, betas=(0.9, 0.999), eps: float = 1e-12,
                 bg=(0.0, 0.0, 0.0)):
        c = camera_from(cam)
        self.params, self.gt, self.lam, self.bg = params, gt.contiguous(), lam, tuple(bg)
        self.intr = (c.fx, c.fy, c.cx, c.cy, c.width, c.height)
        self.R = np.array(list(c.R), np.float64).reshape(3, 3)
        self.t = np.array(list(c.t), np.float64)
        self.vb = ViewBuffers(params.n, c, tiling or tiling_struct(16, 16), 1 << 16)
        self.d_pose = torch.zeros(15, dtype=torch.float32, device=params.mean_op.device)
        self.lr = np.array([lr_trans] * 3 + [lr_rot] * 3)
        self.b1, self.b2, self.eps = betas[0], betas[1], eps
        self.m = np.zeros(6)
        self.v = np.zeros(6)
        self.k = 0

    def camera(self):
        return camera_struct(self.R, self.t, *self.intr)

    def gradient(self):
        """(loss, 15-vector dL/dR, dL/dt, dL/dphi) at the current pose."""
        vb = self.vb
        vb.cam = self.camera()
        ensure_capacity(vb, self.params, self.bg)
        vb.forward(self.params, self.bg)
        vb.loss_fwd_bwd(self.gt, self.lam)
        vb.blend_bwd(bg=self.bg)
        self.d_pose.zero_()
        vb.pose_bwd(self.params, self.d_pose)
        if vb.read_status():
            raise RuntimeError(f"pose refinement: status {vb.read_status():#x}")
        return float(vb.loss.item()), self.d_pose.cpu().numpy().astype(np.float64)

    def step(self) -> float:
        """One Adam step on (rho, phi); returns the loss before it."""
        loss, g = self.gradient()
        tw = np.concatenate([g[9:12], g[12:15]])
        self.k += 1
        self.m = self.b1 * self.m + (1 - self.b1) * tw
        self.v = self.b2 * self.v + (1 - self.b2) * tw * tw
        mh = self.m / (1 - self.b1 ** self.k)
        vh = self.v / (1 - self.b2 ** self.k)
        d = -self.lr * mh / (np.sqrt(vh) + self.eps)
        Q = so3_exp(d[3:])
        self.R = Q @ self.R
        self.t = Q @ self.t + d[:3]
        return loss
