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
    return ok, float((err / bound).max()), group_norms(g, ref)


GROUPS = {"mean": slice(0, 3), "opacity": slice(3, 4), "quat": slice(4, 8), "logscale": slice(8, 11),
          "sh": slice(12, 60)}


def group_norms(g: np.ndarray, ref: np.ndarray) -> dict:
    """Normwise relative error ||g - g*|| / ||g*|| per parameter group ((N, 60)
    layout), or over everything for other shapes."""
    if g.ndim != 2 or g.shape[1] != 60:
        return {"all": float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30))}
    return {k: float(np.linalg.norm((g - ref)[:, s]) / max(np.linalg.norm(ref[:, s]), 1e-30))
            for k, s in GROUPS.items()}


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


# The gradient bar is the plain per-element one, |g - g*| <= max(1e-3 |g*|,
# 1e-6).  An element that misses it is accepted only as a cancellation case:
# its exact value is at most 1 / KAPPA_MIN of C, the sum of its terms'
# magnitudes (kappa = C / |g*| >= KAPPA_MIN, i.e. at least 99 % of the terms
# cancel), and the GPU error stays within the FP32 allowance 2^-15 C.  No more than CANCEL_FRAC_MAX of the checked elements may be such
# cases; each is counted and the worst are printed with their values.
KAPPA_MIN = 100.0
CANCEL_FRAC_MAX = 1e-3


def colour_clamp_waiver(pr: np.ndarray, visible=None, tol: float = 1e-4) -> np.ndarray:
    """(N, 60) mask of the elements a colour-clamp decision can change: for a
    visible Gaussian whose raw colour channel lies within `tol` of the clamp
    at 0 (oracle.project columns 13-15), the SH coefficients of that channel
    and the mean (which enters the colour through the view direction).  FP32
    and FP64 may take that decision differently; every other element of the
    Gaussian, and every element of a culled one (zero on both sides), stays
    checked."""
    near = np.abs(pr[:, 13:16]) < tol
    if visible is not None:
        near &= (np.asarray(visible) > 0)[:, None]
    w = np.zeros((pr.shape[0], 60), bool)
    w[:, 0:3] = near.any(1)[:, None]
    for ch in range(3):
        w[:, 12 + ch:60:3] |= near[:, ch:ch + 1]
    return w


def near_flagged(dec, flagged: np.ndarray, reach: int = 5) -> np.ndarray:
    """(N,) mask of the visible Gaussians whose pixel box comes within `reach`
    pixels of a flagged pixel (a blend decision FP32 and FP64 may take
    differently).  When the upstream gradient is the GPU's own Eq. 4 gradient
    of its own image, a flagged pixel changes dL/dI over its 11 x 11 SSIM
    window (reach 5), so these Gaussians' gradients may differ by more than
    rounding."""
    b = dec.box.astype(np.int64)  # x0, x1, y0, y1, inclusive
    near = np.zeros(b.shape[0], bool)
    for y, x in zip(*np.nonzero(flagged)):
        near |= (b[:, 0] <= x + reach) & (b[:, 1] >= x - reach) & (b[:, 2] <= y + reach) & (b[:, 3] >= y - reach)
    return near & (dec.visible > 0)


def assert_grad_bar(label: str, g: np.ndarray, ref: np.ndarray, cond: np.ndarray, waive=None, rtol=GRAD_RTOL,
                    atol=GRAD_ATOL, max_frac=CANCEL_FRAC_MAX, show: int = 4) -> dict:
    """Asserts the plain per-element gradient bar on every element not waived,
    with the cancellation cases described above as the only exception, and
    prints the error for the result: elements checked, worst err / bar among
    those that meet it, the cancellation cases (count, smallest kappa, largest
    err / C, the worst few with g*, g, C), the waived count and the normwise
    error per group."""
    g, ref, cond = (np.asarray(a, np.float64) for a in (g, ref, cond))
    err = np.abs(g - ref)
    bar = np.maximum(rtol * np.abs(ref), atol)
    checked = np.ones(g.shape, bool) if waive is None else ~np.asarray(waive, bool)
    plain = err <= bar
    fail = checked & ~plain
    kappa = cond / np.maximum(np.abs(ref), 1e-300)
    cancel = fail & (kappa >= KAPPA_MIN) & (err <= GRAD_TAU * cond)
    bad = fail & ~cancel
    n_checked = int(checked.sum())
    met = checked & plain
    rep = {"checked": n_checked, "plain": int(met.sum()), "cancellation": int(cancel.sum()),
           "waived": int((~checked).sum()), "bad": int(bad.sum()),
           "worst_met": float((err / bar)[met].max()) if met.any() else 0.0,
           "normwise": group_norms(g, ref)}
    msg = (f"{label}: {n_checked} elements checked, {rep['plain']} meet |g - g*| <= max(1e-3 |g*|, 1e-6) "
           f"(worst err/bar {rep['worst_met']:.3f}); cancellation cases {rep['cancellation']}")
    if cancel.any():
        msg += (f" (kappa >= {float(kappa[cancel].min()):.0f}, err <= {float((err / cond)[cancel].max()):.2e} C)")
    msg += f"; waived {rep['waived']}; normwise {', '.join(f'{k} {v:.1e}' for k, v in rep['normwise'].items())}"
    for name, sel in (("cancellation", cancel), ("out of tolerance", bad)):
        if sel.any():
            idx = np.argwhere(sel)
            order = np.argsort(-(err / bar)[sel])[:show]
            for j in order:
                ix = tuple(idx[j])
                msg += (f"\n  {name} {ix}: g* {ref[ix]:.6e} g {g[ix]:.6e} err {err[ix]:.2e} C {cond[ix]:.2e} "
                        f"kappa {kappa[ix]:.0f}")
    print(msg)
    assert not bad.any(), f"{label}: {rep['bad']} elements out of tolerance\n{msg}"
    assert rep["cancellation"] <= max_frac * max(n_checked, 1), \
        f"{label}: {rep['cancellation']} cancellation cases exceed {max_frac:g} of {n_checked}"
    return rep


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
