"""FP64 CPU oracle for differentiable 3D-Gaussian rasterisation (Photo-SLAM Sec. 3.3-3.4).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are the only callers.  The product path
(``paper_2311_16728_b300``) never imports this package, and this package never
imports the product.  The C source ``gsr_oracle.c`` holds every formula; this
module only builds it with gcc and marshals numpy arrays through ctypes.

Parameter layout (matches the product's parameter store, as plain memory):
  mean_op  (N, 4)      x, y, z, opacity logit
  quat     (N, 4)      w, x, y, z (unnormalised)
  logscale (N, 4)      3 log-scales + pad
  sh       (12, N, 4)  48 SH floats per Gaussian, coefficient-major (float f is
                       coefficient f // 3, channel f % 3)
Gradients come back as (N, 60): mean xyz, opacity logit, quat wxyz, logscale
xyz, pad, sh[48] in the same coefficient-major order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

NO_CLAMP, NO_SKIP, NO_TERM = 1, 2, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile gsr_oracle.c into oracle/liboracle.so (gcc, FP contraction off)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-D_GNU_SOURCE", "-Wall", "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_num_threads.restype = i32
        L.orc_chain_exp.argtypes = [ctypes.c_float]
        L.orc_chain_exp.restype = ctypes.c_float
        L.orc_sh_basis.argtypes = [P, i32, P, P]
        L.orc_sh_basis.restype = None
        L.orc_decide.argtypes = [i64, P, P, P, P, i32, i32, P, P, P, P, P, P, P]
        L.orc_keys.argtypes = [i64, P, P, P, P, P, P, i32, i32, i32, i32, P, P, i64, P, P]
        L.orc_tile_keep.argtypes = [ctypes.c_float, ctypes.c_float, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float]
        L.orc_tile_keep.restype = i32
        L.orc_render.argtypes = [i64, P, P, P, P, i32, P, i32, i32, P, P, P, P, i32, i32, i32, P, P, P, P]
        L.orc_render_bwd.argtypes = [i64, P, P, P, P, i32, P, i32, i32, P, P, P, P, i32, i32, i32, P, P, P, P]
        L.orc_chain.argtypes = [i64, P, P, P, P, i32, P, i32, i32, P, P, P]
        L.orc_project.argtypes = [i64, P, P, P, P, i32, P, i32, i32, P, P]
        L.orc_ssim_map.argtypes = [P, P, i32, i32, i32, P]
        L.orc_loss.argtypes = [P, P, i32, i32, i32, dbl, P, P]
        L.orc_pyramid_down.argtypes = [P, i32, i32, i32, P]
        L.orc_adam.argtypes = [i64, P, P, P, P, P, i32, dbl, dbl, dbl]
        L.orc_psnr.argtypes = [P, P, i64]
        L.orc_default_init.argtypes = [P, i32, i32, P, i64, P, P, i64, i64, P, P, P, P, P]
        L.orc_densify.argtypes = [i64, P, P, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, i64, P, P, P, P, P]
        L.orc_psnr.restype = dbl
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def chain_exp(x: float) -> float:
    return float(lib().orc_chain_exp(ctypes.c_float(x)))


def sh_basis(v, degree: int = 3):
    """Real SH basis Y[16] and its gradient dY[16, 3] at direction v (FP64)."""
    v = _f64(v)
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().orc_sh_basis(_p(v), int(degree), _p(Y), _p(dY))
    return Y, dY


def camera_array(R, t, fx, fy, cx, cy) -> np.ndarray:
    """16 floats: R (row-major world->camera), t, fx, fy, cx, cy."""
    return _f32(np.concatenate([np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64).reshape(3),
                                [fx, fy, cx, cy]]))


class Decisions:
    """FP32 decision chain outputs: visible, depth, pixel box, uv, radius,
    conic (A, B, C) and opacity."""

    def __init__(self, visible, depth, box, uv, radius, conic, opacity):
        self.visible, self.depth, self.box, self.uv, self.radius = visible, depth, box, uv, radius
        self.conic, self.opacity = conic, opacity


def decide(mean_op, quat, logscale, cam, W: int, H: int) -> Decisions:
    mean_op, quat, logscale, cam = _f32(mean_op), _f32(quat), _f32(logscale), _f32(cam)
    n = mean_op.shape[0]
    vis = np.zeros(n, np.uint8)
    depth = np.zeros(n, np.float32)
    box = np.zeros((n, 4), np.int32)
    uv = np.zeros((n, 2), np.float32)
    rad = np.zeros(n, np.int32)
    conic = np.zeros((n, 3), np.float32)
    op = np.zeros(n, np.float32)
    rc = lib().orc_decide(n, _p(mean_op), _p(quat), _p(logscale), _p(cam), W, H, _p(vis), _p(depth), _p(box),
                          _p(uv), _p(rad), _p(conic), _p(op))
    assert rc == 0
    return Decisions(vis, depth, box, uv, rad, conic, op)


def tile_keep(u, v, conic, opacity, x0, x1, y0, y1) -> bool:
    c = np.ascontiguousarray(conic, np.float32)
    f = ctypes.c_float
    return bool(lib().orc_tile_keep(f(u), f(v), _p(c), f(opacity), f(x0), f(x1), f(y0), f(y1)))


def keys(dec: Decisions, W: int, H: int, tile_w: int = 16, tile_h: int = 16):
    """Sorted (key, gid) pairs of the kept (Gaussian, tile) pairs and per-tile
    ranges (2 * tiles u32)."""
    n = dec.visible.shape[0]
    gx, gy = (W + tile_w - 1) // tile_w, (H + tile_h - 1) // tile_h
    npairs = np.zeros(1, np.int64)
    ranges = np.zeros(2 * gx * gy, np.uint32)
    # first call sizes the pair buffer
    k0 = np.zeros(1, np.uint64)
    v0 = np.zeros(1, np.uint32)
    args = (_p(dec.visible), _p(dec.depth), _p(dec.box), _p(dec.uv), _p(dec.conic), _p(dec.opacity))
    rc = lib().orc_keys(n, *args, W, H, tile_w, tile_h, _p(k0), _p(v0), 0, _p(npairs), _p(ranges))
    cap = int(npairs[0])
    ks = np.zeros(max(cap, 1), np.uint64)
    vs = np.zeros(max(cap, 1), np.uint32)
    rc = lib().orc_keys(n, *args, W, H, tile_w, tile_h, _p(ks), _p(vs), cap, _p(npairs), _p(ranges))
    assert rc == 0
    return ks[:cap], vs[:cap], ranges


class Scene64:
    """FP64 copies of the parameters (exact widening of the FP32 store)."""

    def __init__(self, mean_op, quat, logscale, sh, sh_degree: int = 3):
        self.mean_op = _f64(mean_op)
        self.quat = _f64(quat)
        self.logscale = _f64(logscale)
        self.sh = _f64(sh)
        self.n = self.mean_op.shape[0]
        self.sh_degree = int(sh_degree)
        assert self.sh.shape == (12, self.n, 4)


def render(sc: Scene64, cam, W: int, H: int, dec: Decisions, bg=(0.0, 0.0, 0.0), flags: int = 0,
           rows=None):
    """Returns (img (3,H,W), T_final (H,W), n_contrib (H,W), margin (H,W))."""
    y0, y1 = (0, H) if rows is None else rows
    cam = _f64(cam)
    bg = _f64(bg)
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    mg = np.zeros((H, W))
    rc = lib().orc_render(sc.n, _p(sc.mean_op), _p(sc.quat), _p(sc.logscale), _p(sc.sh), sc.sh_degree, _p(cam), W,
                          H, _p(bg), _p(dec.visible), _p(dec.depth), _p(dec.box), flags, y0, y1, _p(img), _p(T),
                          _p(nc), _p(mg))
    assert rc == 0
    return img, T, nc, mg


def render_bwd(sc: Scene64, cam, W: int, H: int, dec: Decisions, dimg, bg=(0.0, 0.0, 0.0), flags: int = 0,
               rows=None, with_magnitude: bool = False):
    """Returns (grad (N, 60), grad2d (N, 9)) [, grad2d_mag (N, 9)]: the magnitude
    is the per-element sum of |pixel term| (condition scale of each sum)."""
    y0, y1 = (0, H) if rows is None else rows
    cam = _f64(cam)
    bg = _f64(bg)
    dimg = _f64(dimg)
    assert dimg.shape == (3, H, W)
    g = np.zeros((sc.n, 60))
    g2 = np.zeros((sc.n, 9))
    mag = np.zeros((sc.n, 9)) if with_magnitude else None
    rc = lib().orc_render_bwd(sc.n, _p(sc.mean_op), _p(sc.quat), _p(sc.logscale), _p(sc.sh), sc.sh_degree, _p(cam),
                              W, H, _p(bg), _p(dec.visible), _p(dec.depth), _p(dec.box), flags, y0, y1, _p(dimg),
                              _p(g), _p(g2), _p(mag) if with_magnitude else None)
    assert rc == 0
    return (g, g2, mag) if with_magnitude else (g, g2)


def chain(sc: Scene64, cam, W: int, H: int, dec: Decisions, g2):
    cam = _f64(cam)
    g2 = _f64(g2)
    g = np.zeros((sc.n, 60))
    rc = lib().orc_chain(sc.n, _p(sc.mean_op), _p(sc.quat), _p(sc.logscale), _p(sc.sh), sc.sh_degree, _p(cam), W, H,
                         _p(dec.visible), _p(g2), _p(g))
    assert rc == 0
    return g


def pose_grad(sc: Scene64, cam, W: int, H: int, dec: Decisions, g2, with_magnitude: bool = False):
    """Camera pose gradient from the screen-space gradients g2 (N, 9):
    15 values dL/dR (row-major), dL/dt, dL/dphi (left rotation about the
    camera centre) [, and the sums of their per-Gaussian parts' |.|]."""
    cam = _f64(cam)
    g2 = _f64(g2)
    pose = np.zeros(15)
    mag = np.zeros(15)
    rc = lib().orc_pose_grad(sc.n, _p(sc.mean_op), _p(sc.quat), _p(sc.logscale), _p(sc.sh), sc.sh_degree, _p(cam),
                             W, H, _p(dec.visible), _p(g2), _p(pose), _p(mag))
    assert rc == 0
    return (pose, mag) if with_magnitude else pose


def project(sc: Scene64, cam, W: int, H: int, visible):
    """(N, 16): u, v, A, B, C, opacity, r, g, b, depth, a', b', c', raw r, g, b."""
    cam = _f64(cam)
    vis = np.ascontiguousarray(visible, np.uint8)
    out = np.zeros((sc.n, 16))
    rc = lib().orc_project(sc.n, _p(sc.mean_op), _p(sc.quat), _p(sc.logscale), _p(sc.sh), sc.sh_degree, _p(cam), W,
                           H, _p(vis), _p(out))
    assert rc == 0
    return out


def ssim_map(x, y):
    x, y = _f64(x), _f64(y)
    C, H, W = x.shape
    out = np.zeros_like(x)
    lib().orc_ssim_map(_p(x), _p(y), C, H, W, _p(out))
    return out


def loss(x, y, lam: float = 0.2, grad: bool = True):
    """Eq. 4 loss and (optionally) dL/dx."""
    x, y = _f64(x), _f64(y)
    C, H, W = x.shape
    out = np.zeros(1)
    d = np.zeros_like(x) if grad else None
    rc = lib().orc_loss(_p(x), _p(y), C, H, W, float(lam), _p(out), _p(d) if grad else None)
    assert rc == 0
    return (float(out[0]), d) if grad else float(out[0])


def luma(img):
    """Luminance of a 3 x H x W image (BT.601 weights, the reading for the
    grayscale views): 0.299 R + 0.587 G + 0.114 B, as 1 x H x W (FP64)."""
    img = _f64(img)
    return (0.299 * img[0] + 0.587 * img[1] + 0.114 * img[2])[None]


def pyramid_down(img):
    img = _f64(img)
    C, H, W = img.shape
    out = np.zeros((C, (H + 1) // 2, (W + 1) // 2))
    lib().orc_pyramid_down(_p(img), C, H, W, _p(out))
    return out


def adam(p, g, m, v, lr, step: int, b1=0.9, b2=0.999, eps=1e-15):
    """In-place Adam update of FP64 copies; returns (p, m, v)."""
    p, g, m, v, lr = _f64(p).copy(), _f64(g), _f64(m).copy(), _f64(v).copy(), _f64(lr)
    rc = lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), _p(lr), int(step), b1, b2, eps)
    assert rc == 0
    return p, m, v


def psnr(img, gt) -> float:
    img, gt = _f64(img), _f64(gt)
    return float(lib().orc_psnr(_p(img), _p(gt), img.size))


def default_init(img, keypoints, cam, ref_xyz, offset: int):
    """Default initialisation of M new primitives (see orc_default_init).
    keypoints (M, 5) float32; ref_xyz (N, 3) map means, rows offset ..
    offset + M - 1 being the new primitives.  Returns a dict of FP64 arrays:
    mean (M,3), logscale (M,3), quat (M,4), logit (M,), sh (M,48)."""
    img = _f64(img)
    C, H, W = img.shape
    kp = np.ascontiguousarray(keypoints, np.float32)
    M = kp.shape[0]
    ref = _f64(ref_xyz)
    out = {"mean": np.zeros((M, 3)), "logscale": np.zeros((M, 3)), "quat": np.zeros((M, 4)),
           "logit": np.zeros(M), "sh": np.zeros((M, 48))}
    rc = lib().orc_default_init(_p(img), W, H, _p(kp), M, _p(_f32(cam)), _p(ref), ref.shape[0], int(offset),
                                _p(out["mean"]), _p(out["logscale"]), _p(out["quat"]), _p(out["logit"]), _p(out["sh"]))
    assert rc == 0
    return out


def densify(mean_op, quat, logscale, stat, count, eps, grad_thr, logit_min, logscale_split, shrink):
    """Densification decisions and outputs (see orc_densify).  Returns a dict:
    src (n_out,), kind (n_out,), mean (n_out, 3), logscale (n_out, 3)."""
    mo, q, ls = _f32(mean_op), _f32(quat), _f32(logscale)
    n = mo.shape[0]
    cap = 2 * n
    n_out = np.zeros(1, np.int64)
    src = np.zeros(max(cap, 1), np.int64)
    kind = np.zeros(max(cap, 1), np.int32)
    mean = np.zeros((max(cap, 1), 3))
    lso = np.zeros((max(cap, 1), 3))
    rc = lib().orc_densify(n, _p(mo), _p(q), _p(ls), _p(_f32(stat)), _p(_f32(count)), _p(_f32(eps)),
                           float(grad_thr), float(logit_min), float(logscale_split), float(shrink), cap, _p(n_out),
                           _p(src), _p(kind), _p(mean), _p(lso))
    assert rc == 0
    k = int(n_out[0])
    return {"src": src[:k], "kind": kind[:k], "mean": mean[:k], "logscale": lso[:k]}


def grad_to_planes(g60: np.ndarray):
    """(N, 60) oracle gradient -> (mean_op (N,4), quat (N,4), logscale (N,4), sh (12,N,4))."""
    n = g60.shape[0]
    return (g60[:, 0:4], g60[:, 4:8], g60[:, 8:12], np.ascontiguousarray(g60[:, 12:60].reshape(n, 12, 4).transpose(1, 0, 2)))
