"""Shared plumbing for the GPU-vs-oracle parity tests (inputs come from
`synthetic`, expected values from `oracle`; nothing here computes the method)."""
from __future__ import annotations

import numpy as np

import oracle
import synthetic as S

# Tolerances (stated per result by the tests):
IMG_ATOL = 1e-4           # rendered image, max abs on [0, 1]
GRAD_RTOL = 1e-3          # gradients: |g - g*| <= max(GRAD_RTOL |g*|, GRAD_ATOL)
GRAD_ATOL = 1e-6
MARGIN_FLAG = 1e-5        # oracle decision margin below which FP32 and FP64 may disagree
# FP32 allowance for gradient sums with cancellation: each term passes through
# a few dozen rounded FP32 operations and the transmittance recovery
# T_i = T_{i+1} / (1 - alpha_i) amplifies the relative error of (1 - alpha_i)
# by alpha / (1 - alpha) <= 99, so a sum may be off by ~1e-5 of the sum of its
# |terms| even when the exact value is tiny.  2^-15 = 512 FP32 ulps.
GRAD_TAU = 2.0 ** -15


def oracle_scene(p: S.Params, sh_degree: int = 3):
    return oracle.Scene64(p.mean_op, p.quat, p.logscale, p.sh, sh_degree)


def to_gpu(p: S.Params, sh_degree: int = 3):
    import paper_2311_16728_b300 as gsr
    return gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh, sh_degree)


def gpu_view(p: S.Params, cam: S.Camera, tile=(16, 16), sh_degree: int = 3, cap=None, bg=(0.0, 0.0, 0.0)):
    """Runs preprocess -> bin/sort -> render on the GPU; returns (ViewBuffers, Gaussians)."""
    import paper_2311_16728_b300 as gsr
    g = to_gpu(p, sh_degree)
    vb = gsr.ViewBuffers(p.n, gsr.camera_from(cam), gsr.tiling_struct(*tile), cap or max(1024, 64 * p.n))
    if cap is None:
        gsr.ensure_capacity(vb, g, bg)
    vb.forward(g, bg)
    import torch
    torch.cuda.synchronize()
    return vb, g


def unpack_box(c_op_box: np.ndarray) -> np.ndarray:
    bx = c_op_box[:, 2].view(np.uint32)
    by = c_op_box[:, 3].view(np.uint32)
    return np.stack([bx & 0xFFFF, bx >> 16, by & 0xFFFF, by >> 16], 1).astype(np.int32)


def grad_planes_gpu(grads) -> np.ndarray:
    """GPU gradient store -> (N, 60) in the oracle's layout."""
    n = grads.n
    mo = grads.mean_op.cpu().numpy()
    q = grads.quat.cpu().numpy()
    ls = grads.logscale.cpu().numpy()
    sh = grads.sh.cpu().numpy().transpose(1, 0, 2).reshape(n, 48)
    return np.concatenate([mo, q, ls, sh], 1).astype(np.float64)


def grad_report(g: np.ndarray, ref: np.ndarray, rtol=GRAD_RTOL, atol=GRAD_ATOL):
    """Per-element pass mask, worst excess and normwise relative error per group."""
    err = np.abs(g - ref)
    bound = np.maximum(rtol * np.abs(ref), atol)
    ok = err <= bound
    groups = {"mean": slice(0, 3), "opacity": slice(3, 4), "quat": slice(4, 8), "logscale": slice(8, 11),
              "sh": slice(12, 60)}
    norms = {k: float(np.linalg.norm((g - ref)[:, s]) / max(np.linalg.norm(ref[:, s]), 1e-30))
             for k, s in groups.items()}
    return ok, float((err / bound).max()), norms


def param_condition(sc, cam_arr, W, H, dec, mag2d):
    """Condition magnitude of every parameter-gradient element: the screen-space
    magnitudes pushed through the absolute value of the per-Gaussian chain
    Jacobian (sum_k |d g_param / d g2d_k| * mag2d_k), from the oracle."""
    n = sc.n
    C = np.zeros((n, 60))
    for k in range(9):
        e = np.zeros((n, 9))
        e[:, k] = 1.0
        C += np.abs(oracle.chain(sc, cam_arr, W, H, dec, e)) * mag2d[:, k:k + 1]
    return C


def grad_check(g: np.ndarray, ref: np.ndarray, cond: np.ndarray, rtol=GRAD_RTOL, atol=GRAD_ATOL, tau=None):
    """Per-element bar |g - g*| <= max(rtol |g*|, atol) + tau * cond.

    cond is the element's condition magnitude (sum of |terms|); tau covers the
    FP32 evaluation of each term and of the sum.  Returns (ok mask, number of
    elements that needed the tau allowance, worst ratio err / bound)."""
    tau = GRAD_TAU if tau is None else tau
    err = np.abs(g - ref)
    base = np.maximum(rtol * np.abs(ref), atol)
    bound = base + tau * cond
    return err <= bound, int(((err > base) & (err <= bound)).sum()), float((err / bound).max())


def morton_codes(mean, lo, hi):
    """30-bit Morton codes of the means as the store-order kernel forms them:
    each coordinate quantised to 10 bits (FP32 (v - lo) * (1024 / (hi - lo)),
    clamped to [0, 1023], truncated), the bits interleaved x, y, z from bit 0
    up."""
    lo32, hi32 = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    q = []
    for k in range(3):
        s = np.float32(1024.0) / (hi32[k] - lo32[k])
        t = (mean[:, k].astype(np.float32) - lo32[k]) * s
        q.append(np.clip(t, 0.0, 1023.0).astype(np.uint32))
    code = np.zeros(mean.shape[0], np.uint64)
    for b in range(10):
        for k in range(3):
            code |= ((q[k].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + k)
    return code


def morton_permuted(p: S.Params, lo, hi) -> S.Params:
    """The parameter set in the store order the benchmark uses (stable sort
    by Morton code of the means), computed on the host."""
    perm = np.lexsort((np.arange(p.n), morton_codes(p.mean_op[:, :3], lo, hi)))
    return S.Params(p.mean_op[perm], p.quat[perm], p.logscale[perm], p.sh[:, perm])
