"""FP64 oracle of the learned initialiser MLP (TEST INFRASTRUCTURE ONLY).

Photo-SLAM densifies new hyper primitives at inactive ORB keypoints (Sec.
3.3.1, geometry-based densification); the paper does not say how their
rotation, scaling, density and SH are initialised.  The build's learned
initialiser is a small MLP mapping a keypoint's image patches to those
parameters:

  x   = [3 pyramid levels x 16 x 16 x RGB (2304), depth, log scale, cos th, sin th]
        (2308 values, zero-padded to K0 = 2368)
  h1  = relu(W1 x + b1)            256
  h2  = relu(W2 h1 + b2)           256
  y   = W3 h2 + b3                 56 (padded to 64): log-scale 3, quat 4,
                                   opacity logit 1, SH 48
  L   = sum_{m, j < 56} w_j (y_mj - t_mj)^2 / M      (mean squared error)

The GPU computes the products of BF16 operands with FP32 accumulation; this
oracle rounds the same operands to BF16 (round to nearest even) at the same
places, then works in FP64, so the only difference left is the GPU's FP32
summation order, bounded by K 2^-24 sum |a b|.  Nothing here is imported by
the product, and nothing of the product is imported here.
"""
from __future__ import annotations

import numpy as np

K_IN = 2308
K0 = 2368          # K_IN padded to a multiple of 64
H = 256
N_OUT = 56
N3 = 64            # N_OUT padded


def bf16_round(a) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, np.float32)
    shape = f.shape
    f = f.reshape(-1)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[np.isnan(f)] = np.nan
    return out.reshape(shape)


def forward(params, x, *, round_bf16: bool = True):
    """params: dict W1 (H, K0), b1 (H,), W2 (H, H), b2, W3 (N3, H), b3 (N3,).
    x: (M, K0).  Returns dict of the intermediate values (FP64)."""
    rnd = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    xb = rnd(x)
    W1, W2, W3 = rnd(params["W1"]), rnd(params["W2"]), rnd(params["W3"])
    pre1 = xb @ W1.T + np.asarray(params["b1"], np.float64)
    h1 = np.maximum(pre1, 0.0)
    h1b = rnd(h1)
    pre2 = h1b @ W2.T + np.asarray(params["b2"], np.float64)
    h2 = np.maximum(pre2, 0.0)
    h2b = rnd(h2)
    y = h2b @ W3.T + np.asarray(params["b3"], np.float64)
    return {"xb": xb, "W1": W1, "W2": W2, "W3": W3, "pre1": pre1, "h1": h1b, "pre2": pre2, "h2": h2b, "y": y}


def loss_and_dy(y, target, weight):
    """MSE over the first N_OUT outputs (weights per output), gradient dL/dy
    (padding columns get zero)."""
    M = y.shape[0]
    d = (y[:, :N_OUT] - target[:, :N_OUT]) * weight[None, :N_OUT]
    L = float(np.sum(d * (y[:, :N_OUT] - target[:, :N_OUT])) / M)
    dy = np.zeros_like(y)
    dy[:, :N_OUT] = 2.0 * d / M
    return L, dy


def backward(fw, dy, *, round_bf16: bool = True):
    """Gradients of the loss w.r.t. W1, b1, W2, b2, W3, b3 given dL/dy.
    dy and the back-propagated activation gradients are rounded to BF16 where
    the GPU feeds them to a BF16 GEMM."""
    rnd = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    dyb = rnd(dy)
    gW3 = dyb.T @ fw["h2"]
    gb3 = dy.sum(0)
    dh2 = dyb @ fw["W3"]
    dpre2 = dh2 * (fw["pre2"] > 0)
    dpre2b = rnd(dpre2)
    gW2 = dpre2b.T @ fw["h1"]
    gb2 = dpre2.sum(0)
    dh1 = dpre2b @ fw["W2"]
    dpre1 = dh1 * (fw["pre1"] > 0)
    dpre1b = rnd(dpre1)
    gW1 = dpre1b.T @ fw["xb"]
    gb1 = dpre1.sum(0)
    return {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def init_params(seed: int = 3):
    """He-uniform weights, zero biases (FP32 master copies)."""
    rng = np.random.default_rng(seed)

    def lin(out, fan_in, rows, cols):
        w = np.zeros((rows, cols), np.float32)
        lim = np.sqrt(6.0 / fan_in)
        w[:out, :fan_in] = rng.uniform(-lim, lim, (out, fan_in))
        return w

    return {"W1": lin(H, K_IN, H, K0), "b1": np.zeros(H, np.float32), "W2": lin(H, H, H, H),
            "b2": np.zeros(H, np.float32), "W3": lin(N_OUT, H, N3, H), "b3": np.zeros(N3, np.float32)}
