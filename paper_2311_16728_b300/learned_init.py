"""Learned initialiser of new primitives (torch glue over the gsr_mlp_* calls).

Photo-SLAM creates extra primitives at inactive ORB keypoints (Sec. 3.3.1,
geometry-based densification) without saying how they are initialised.
Here a 2308 -> 256 -> 256 -> 56 MLP predicts each new primitive's log-scale,
rotation, opacity and SH from the keypoint's three-level image patches,
depth, scale and angle; it runs and trains on the tensor cores (BF16
operands, FP32 accumulation, FP32 master weights).  `default_init` is the
fallback used without it.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from .raster import Gaussians, _p, _stream, camera_from

K_IN, K0, H, N_OUT, N3 = 2308, 2368, 256, 56, 64


def pad_rows(m: int) -> int:
    return max(128, (m + 127) // 128 * 128)


def init_weights(seed: int = 3) -> dict:
    """He-uniform FP32 weights (limit sqrt(6 / fan_in)) on the valid block of
    each layer, zero padding and zero biases."""
    rng = np.random.default_rng(seed)

    def layer(rows_valid, fan_in, rows, cols):
        w = np.zeros((rows, cols), np.float32)
        bound = np.sqrt(6.0 / fan_in)
        w[:rows_valid, :fan_in] = rng.uniform(-bound, bound, (rows_valid, fan_in))
        return w

    return {"W1": layer(H, K_IN, H, K0), "b1": np.zeros(H, np.float32), "W2": layer(H, H, H, H),
            "b2": np.zeros(H, np.float32), "W3": layer(N_OUT, H, N3, H), "b3": np.zeros(N3, np.float32)}


class MLPWeights:
    """FP32 masters + BF16 copies (or FP32-only moments) on the device."""

    def __init__(self, arrays=None, device="cuda", with_half=True):
        shapes = {"W1": (H, K0), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (N3, H), "b3": (N3,)}
        self.t = {k: (torch.as_tensor(np.asarray(arrays[k]), dtype=torch.float32, device=device).contiguous()
                      if arrays is not None else torch.zeros(s, dtype=torch.float32, device=device))
                  for k, s in shapes.items()}
        self.h = {}
        if with_half:
            bf = dict(dtype=torch.bfloat16, device=device)
            self.h = {"W1h": torch.empty(H, K0, **bf), "W2h": torch.empty(H, H, **bf),
                      "W2hT": torch.empty(H, H, **bf), "W3h": torch.empty(N3, H, **bf),
                      "W3hT": torch.empty(H, N3, **bf)}

    def struct(self) -> L.gsr_mlp_weights:
        s = L.gsr_mlp_weights(*(self.t[k].data_ptr() for k in ("W1", "b1", "W2", "b2", "W3", "b3")))
        for k, v in self.h.items():
            setattr(s, k, v.data_ptr())
        return s

    def sync(self, stream=None):
        s = self.struct()
        L.gsr_mlp_sync_weights(ctypes.byref(s), _stream(stream))


def default_init(map_params: Gaussians, img0: torch.Tensor, keypoints: torch.Tensor, cam, offset: int,
                 stream=None):
    """The fallback initialiser: writes Gaussians offset .. offset + M - 1 of
    `map_params` from keypoints (M, 5) = (u, v, depth, log scale, angle) seen in
    `cam` with level-0 image img0 (3, H, W)."""
    M = keypoints.shape[0]
    sz = ctypes.c_size_t()
    L.gsr_default_init_workspace_size(M, map_params.n, ctypes.byref(sz))
    ws = torch.empty(sz.value, dtype=torch.uint8, device=img0.device)
    c, o = camera_from(cam), map_params.buffers_struct()
    _, H0, W0 = img0.shape
    L.gsr_default_init(_p(img0.contiguous()), W0, H0, _p(keypoints.contiguous()), M, ctypes.byref(c), ctypes.byref(o),
                       map_params.n, offset, _p(ws), ws.numel(), _stream(stream))


class LearnedInit:
    def __init__(self, weights: dict, batch_capacity: int, lr: float = 1e-3, device="cuda"):
        self.w = MLPWeights(weights, device)
        self.m = MLPWeights(None, device, with_half=False)
        self.v = MLPWeights(None, device, with_half=False)
        self.w.sync()
        self.mpad = pad_rows(batch_capacity)
        sz = ctypes.c_size_t()
        L.gsr_mlp_workspace_size(self.mpad, ctypes.byref(sz))
        self.ws = torch.empty(sz.value, dtype=torch.uint8, device=device)
        bf = dict(dtype=torch.bfloat16, device=device)
        self.x = torch.zeros(self.mpad, K0, **bf)
        self.xT = torch.zeros(K0, self.mpad, **bf)
        self.y = torch.zeros(self.mpad, N3, dtype=torch.float32, device=device)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.lr = lr
        self.out_weight = torch.ones(N3, dtype=torch.float32, device=device)
        self.out_weight[N_OUT:] = 0

    def gather(self, levels, keypoints: torch.Tensor, transpose: bool, stream=None):
        """levels: [GP^0, GP^1, GP^2] (3 x H_l x W_l); keypoints (M, 5)."""
        M = keypoints.shape[0]
        assert M <= self.mpad
        _, H0, W0 = levels[0].shape
        L.gsr_patch_gather(_p(levels[0]), _p(levels[1]), _p(levels[2]), W0, H0, _p(keypoints.contiguous()), M,
                           self.mpad, _p(self.x), _p(self.xT) if transpose else None, _stream(stream))
        return M

    def forward(self, stream=None) -> torch.Tensor:
        s = self.w.struct()
        L.gsr_mlp_forward(ctypes.byref(s), _p(self.x), self.mpad, _p(self.y), _p(self.ws), self.ws.numel(),
                          _p(self.status), _stream(stream))
        return self.y

    def train_step(self, target: torch.Tensor, M: int, stream=None, x: torch.Tensor = None, xT: torch.Tensor = None):
        """One training step on rows 0 .. M - 1 of x (default: the gather
        buffers; any [Mpad, 2368] BF16 input with its transpose)."""
        w, m, v = self.w.struct(), self.m.struct(), self.v.struct()
        x = self.x if x is None else x
        xT = self.xT if xT is None else xT
        assert x.shape == self.x.shape and xT.shape == self.xT.shape
        L.gsr_mlp_train_step(ctypes.byref(w), ctypes.byref(m), ctypes.byref(v), _p(x), _p(xT),
                             _p(target), _p(self.out_weight), M, self.mpad, self.lr, 0.9, 0.999, 1e-8,
                             _p(self.step_count), _p(self.loss), _p(self.y), _p(self.ws), self.ws.numel(),
                             _p(self.status), _stream(stream))

    def gradients(self) -> dict:
        g = L.gsr_mlp_weights()
        L.gsr_mlp_gradients(_p(self.ws), self.mpad, ctypes.byref(g))
        out = {}
        for k, shape in (("W1", (H, K0)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, N3)),
                         ("b3", (N3,))):
            n = int(np.prod(shape))
            ptr = getattr(g, k)
            base = self.ws.data_ptr()
            off = (ptr - base) // 4
            out[k] = self.ws.view(torch.float32)[off:off + n].view(*shape)
        out["W3"] = out["W3"].t()  # stored transposed
        return out

    def encode_targets(self, g: Gaussians, gids: torch.Tensor, keypoints: torch.Tensor, cam, target: torch.Tensor,
                       stream=None, base: torch.Tensor = None):
        """Encoded parameters of Gaussians gids[m] (minus `base` rows if given)."""
        gs, c = g.gaussians_struct(), camera_from(cam)
        L.gsr_mlp_encode_targets(ctypes.byref(gs), _p(gids), _p(keypoints), keypoints.shape[0], self.mpad,
                                 ctypes.byref(c), _p(base), _p(target), _stream(stream))

    def decode(self, keypoints: torch.Tensor, cam, out: Gaussians, offset: int, stream=None,
               base: torch.Tensor = None):
        """Writes Gaussians offset .. offset + M - 1 from y (+ `base`)."""
        c, o = camera_from(cam), out.buffers_struct()
        L.gsr_mlp_decode(_p(self.y), _p(base), _p(keypoints), keypoints.shape[0], ctypes.byref(c), ctypes.byref(o),
                         out.n, offset, _stream(stream))
