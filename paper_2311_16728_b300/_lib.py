"""ctypes binding of libgsr.so: the C ABI declared in include/gsr.h, name for name.

Argument marshalling only -- every step of the hot path runs in the CUDA
kernels behind these calls.  There is no fallback: if the shared library is
missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_size_t, c_void_p

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgsr.so")

GSR_OK = 0
GSR_ERR_INVALID_ARG = 1
GSR_ERR_CAPACITY = 2
GSR_ERR_CUDA = 3
GSR_ERR_TIMEOUT = 4
GSR_ERR_UNSUPPORTED = 5
STATUS_NAMES = {0: "GSR_OK", 1: "GSR_ERR_INVALID_ARG", 2: "GSR_ERR_CAPACITY", 3: "GSR_ERR_CUDA",
                4: "GSR_ERR_TIMEOUT", 5: "GSR_ERR_UNSUPPORTED"}


class gsr_gaussians(ctypes.Structure):
    _fields_ = [("mean_op", c_void_p), ("quat", c_void_p), ("logscale", c_void_p), ("sh", c_void_p),
                ("n", c_int64), ("sh_degree", c_int32)]


class gsr_param_buffers(ctypes.Structure):
    _fields_ = [("mean_op", c_void_p), ("quat", c_void_p), ("logscale", c_void_p), ("sh", c_void_p)]


class gsr_camera(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int32), ("height", c_int32)]


class gsr_tiling(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch_depth", c_int32), ("bwd_threads", c_int32)]


class gsr_proj(ctypes.Structure):
    _fields_ = [("xy_conic", c_void_p), ("c_op_box", c_void_p), ("rgb_depth", c_void_p), ("ntiles", c_void_p),
                ("uv_lo", c_void_p), ("tile_order", c_void_p),
                ("tile_work", c_void_p)]


class gsr_grad2d(ctypes.Structure):
    _fields_ = [("g0", c_void_p), ("g1", c_void_p), ("g2", c_void_p)]


class gsr_mlp_weights(ctypes.Structure):
    _fields_ = [("W1", c_void_p), ("b1", c_void_p), ("W2", c_void_p), ("b2", c_void_p), ("W3", c_void_p),
                ("b3", c_void_p), ("W1h", c_void_p), ("W2h", c_void_p), ("W2hT", c_void_p), ("W3h", c_void_p),
                ("W3hT", c_void_p)]


class gsr_densify_config(ctypes.Structure):
    _fields_ = [("grad_thr", c_float), ("logit_min", c_float), ("logscale_split", c_float), ("shrink", c_float)]


class gsr_adam_config(ctypes.Structure):
    _fields_ = [("lr_mean", c_float), ("lr_opacity", c_float), ("lr_quat", c_float), ("lr_scale", c_float),
                ("lr_sh", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float)]


P = POINTER
# gsr_autotune_fn: (candidate, action, ctx) -> status
AUTOTUNE_FN = ctypes.CFUNCTYPE(c_int32, c_int32, c_int32, c_void_p)
GSR_AUTOTUNE_SETUP, GSR_AUTOTUNE_STEP, GSR_AUTOTUNE_RELEASE = 0, 1, 2
_SIGNATURES = {
    "gsr_version": ([], c_char_p),
    "gsr_last_error": ([], c_char_p),
    "gsr_status_read": ([c_void_p, P(c_int32), c_void_p], c_int32),
    "gsr_camera_at_level": ([P(gsr_camera), c_int32, P(gsr_camera)], c_int32),
    "gsr_preprocess": ([P(gsr_gaussians), P(gsr_camera), P(gsr_tiling), P(gsr_proj), c_void_p, c_void_p], c_int32),
    "gsr_bin_sort_workspace_size": ([c_int64, c_int64, P(gsr_camera), P(gsr_tiling), P(c_size_t)], c_int32),
    "gsr_bin_sort": ([P(gsr_proj), c_int64, P(gsr_camera), P(gsr_tiling), c_void_p, c_void_p, c_int64, c_void_p,
                      c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "gsr_render_fwd": ([P(gsr_proj), c_void_p, c_void_p, P(gsr_camera), P(gsr_tiling), c_void_p, c_void_p,
                        c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "gsr_blend_bwd": ([P(gsr_proj), c_int64, c_void_p, c_void_p, P(gsr_camera), P(gsr_tiling), c_void_p, c_void_p,
                       c_void_p, c_void_p, P(gsr_grad2d), c_void_p], c_int32),
    "gsr_preprocess_bwd": ([P(gsr_gaussians), P(gsr_proj), P(gsr_camera), P(gsr_tiling), P(gsr_grad2d),
                            P(gsr_param_buffers), c_void_p, c_void_p, c_void_p], c_int32),
    "gsr_autotune": ([c_int32, AUTOTUNE_FN, c_void_p, c_int32, c_int32, c_void_p, P(c_float), P(c_int32)], c_int32),
    "gsr_spatial_order_workspace_size": ([c_int64, P(c_size_t)], c_int32),
    "gsr_spatial_order": ([P(gsr_gaussians), c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
    "gsr_permute": ([P(gsr_param_buffers), P(gsr_param_buffers), c_void_p, c_int64, c_void_p], c_int32),
    "gsr_pose_bwd": ([P(gsr_gaussians), P(gsr_proj), P(gsr_camera), P(gsr_tiling), P(gsr_grad2d), c_void_p,
                      c_void_p], c_int32),
    "gsr_preprocess_bwd_store": ([P(gsr_gaussians), P(gsr_proj), P(gsr_camera), P(gsr_tiling), P(gsr_grad2d),
                            P(gsr_param_buffers), c_void_p, c_void_p, c_void_p], c_int32),
    "gsr_loss_workspace_size": ([c_int32, c_int32, c_int32, P(c_size_t)], c_int32),
    "gsr_loss_luma_workspace_size": ([c_int32, c_int32, P(c_size_t)], c_int32),
    "gsr_loss_luma_fwd_bwd": ([c_void_p, c_void_p, c_int32, c_int32, c_float, c_void_p, c_void_p, c_void_p, c_size_t,
                               c_void_p], c_int32),
    "gsr_loss_fwd_bwd": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p, c_void_p,
                          c_size_t, c_void_p], c_int32),
    "gsr_loss_fwd_bwd_static": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p,
                                 c_void_p], c_int32),
    "gsr_render_bwd": ([P(gsr_gaussians), P(gsr_proj), c_void_p, c_void_p, P(gsr_camera), P(gsr_tiling), c_void_p,
                        c_void_p, c_void_p, c_void_p, P(gsr_grad2d), P(gsr_param_buffers), c_void_p, c_void_p,
                        c_void_p], c_int32),
    "gsr_batched_preprocess": ([P(gsr_gaussians), c_void_p, c_int32, P(gsr_tiling), P(gsr_proj), c_void_p], c_int32),
    "gsr_batched_bin_sort": ([P(gsr_proj), c_int64, c_void_p, c_int32, P(gsr_tiling), c_void_p, c_void_p, c_int64,
                              c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "gsr_batched_iterate_workspace_size": ([c_void_p, c_int32, P(c_size_t)], c_int32),
    "gsr_batched_iterate": ([P(gsr_proj), c_void_p, c_void_p, c_void_p, c_int32, P(gsr_tiling), c_void_p, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p, P(gsr_grad2d),
                             c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "gsr_batched_preprocess_bwd": ([P(gsr_gaussians), P(gsr_proj), c_void_p, c_void_p, c_int32, P(gsr_tiling),
                                    P(gsr_grad2d), P(gsr_param_buffers), c_void_p, c_void_p], c_int32),
    "gsr_default_init_workspace_size": ([c_int64, c_int64, P(c_size_t)], c_int32),
    "gsr_default_init": ([c_void_p, c_int32, c_int32, c_void_p, c_int64, P(gsr_camera), P(gsr_param_buffers), c_int64,
                          c_int64, c_void_p, c_size_t, c_void_p], c_int32),
    "gsr_densify_workspace_size": ([c_int64, P(c_size_t)], c_int32),
    "gsr_densify": ([P(gsr_param_buffers), P(gsr_param_buffers), P(gsr_param_buffers), c_int64, c_void_p, c_void_p,
                     c_void_p, P(gsr_densify_config), P(gsr_param_buffers), P(gsr_param_buffers),
                     P(gsr_param_buffers), c_int64, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "gsr_gemm_bf16": ([c_void_p, c_int64, c_void_p, c_int64, c_int32, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                       c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_int32, c_void_p, c_int64,
                       c_int32, c_void_p, c_void_p], c_int32),
    "gsr_mlp_workspace_size": ([c_int64, P(c_size_t)], c_int32),
    "gsr_mlp_sync_weights": ([P(gsr_mlp_weights), c_void_p], c_int32),
    "gsr_patch_gather": ([c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int64, c_int64, c_void_p,
                          c_void_p, c_void_p], c_int32),
    "gsr_mlp_forward": ([P(gsr_mlp_weights), c_void_p, c_int64, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p],
                        c_int32),
    "gsr_mlp_train_step": ([P(gsr_mlp_weights), P(gsr_mlp_weights), P(gsr_mlp_weights), c_void_p, c_void_p, c_void_p,
                            c_void_p, c_int64, c_int64, c_float, c_float, c_float, c_float, c_void_p, c_void_p,
                            c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], c_int32),
    "gsr_mlp_gradients": ([c_void_p, c_int64, P(gsr_mlp_weights)], c_int32),
    "gsr_mlp_encode_targets": ([P(gsr_gaussians), c_void_p, c_void_p, c_int64, c_int64, P(gsr_camera), c_void_p,
                                c_void_p, c_void_p], c_int32),
    "gsr_mlp_decode": ([c_void_p, c_void_p, c_void_p, c_int64, P(gsr_camera), P(gsr_param_buffers), c_int64,
                        c_int64, c_void_p], c_int32),
    "gsr_adam_step": ([P(gsr_param_buffers), P(gsr_param_buffers), P(gsr_param_buffers), P(gsr_param_buffers),
                       c_int64, P(gsr_adam_config), c_void_p, c_void_p], c_int32),
    "gsr_adam_step_touched": ([P(gsr_param_buffers), P(gsr_param_buffers), P(gsr_param_buffers), P(gsr_param_buffers),
                               c_int64, P(gsr_adam_config), c_void_p, c_void_p, c_void_p], c_int32),
    "gsr_pyramid_down": ([c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p], c_int32),
    "gsr_psnr_workspace_size": ([c_int64, P(c_size_t)], c_int32),
    "gsr_psnr": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_size_t, c_void_p], c_int32),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgsr.so not built ({LIB_PATH}); run paper_2311_16728_b300/_build.py or "
                          "__graft_entry__.build() -- there is no non-CUDA fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


class GsrError(RuntimeError):
    def __init__(self, name: str, code: int):
        msg = LIB.gsr_last_error().decode()
        super().__init__(f"{name} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _wrap(name):
    f = getattr(LIB, name)

    def call(*args):
        rc = f(*args)
        if rc != GSR_OK:
            raise GsrError(name, rc)
        return rc

    call.__name__ = name
    call.raw = f
    return call


gsr_version = LIB.gsr_version
gsr_last_error = LIB.gsr_last_error
gsr_status_read = _wrap("gsr_status_read")
gsr_camera_at_level = _wrap("gsr_camera_at_level")
gsr_preprocess = _wrap("gsr_preprocess")
gsr_bin_sort_workspace_size = _wrap("gsr_bin_sort_workspace_size")
gsr_bin_sort = _wrap("gsr_bin_sort")
gsr_render_fwd = _wrap("gsr_render_fwd")
gsr_blend_bwd = _wrap("gsr_blend_bwd")
gsr_preprocess_bwd = _wrap("gsr_preprocess_bwd")
gsr_preprocess_bwd_store = _wrap("gsr_preprocess_bwd_store")
gsr_pose_bwd = _wrap("gsr_pose_bwd")
gsr_autotune = _wrap("gsr_autotune")
gsr_spatial_order_workspace_size = _wrap("gsr_spatial_order_workspace_size")
gsr_spatial_order = _wrap("gsr_spatial_order")
gsr_permute = _wrap("gsr_permute")
gsr_loss_workspace_size = _wrap("gsr_loss_workspace_size")
gsr_loss_fwd_bwd = _wrap("gsr_loss_fwd_bwd")
gsr_loss_fwd_bwd_static = _wrap("gsr_loss_fwd_bwd_static")
gsr_render_bwd = _wrap("gsr_render_bwd")
gsr_batched_preprocess = _wrap("gsr_batched_preprocess")
gsr_batched_bin_sort = _wrap("gsr_batched_bin_sort")
gsr_batched_iterate_workspace_size = _wrap("gsr_batched_iterate_workspace_size")
gsr_batched_iterate = _wrap("gsr_batched_iterate")
gsr_batched_preprocess_bwd = _wrap("gsr_batched_preprocess_bwd")
gsr_default_init_workspace_size = _wrap("gsr_default_init_workspace_size")
gsr_default_init = _wrap("gsr_default_init")
gsr_densify_workspace_size = _wrap("gsr_densify_workspace_size")
gsr_densify = _wrap("gsr_densify")
gsr_gemm_bf16 = _wrap("gsr_gemm_bf16")
gsr_mlp_workspace_size = _wrap("gsr_mlp_workspace_size")
gsr_mlp_sync_weights = _wrap("gsr_mlp_sync_weights")
gsr_patch_gather = _wrap("gsr_patch_gather")
gsr_mlp_forward = _wrap("gsr_mlp_forward")
gsr_mlp_train_step = _wrap("gsr_mlp_train_step")
gsr_mlp_gradients = _wrap("gsr_mlp_gradients")
gsr_mlp_encode_targets = _wrap("gsr_mlp_encode_targets")
gsr_mlp_decode = _wrap("gsr_mlp_decode")
gsr_adam_step = _wrap("gsr_adam_step")
gsr_adam_step_touched = _wrap("gsr_adam_step_touched")
gsr_pyramid_down = _wrap("gsr_pyramid_down")
gsr_psnr_workspace_size = _wrap("gsr_psnr_workspace_size")
gsr_psnr = _wrap("gsr_psnr")
gsr_loss_luma_workspace_size = _wrap("gsr_loss_luma_workspace_size")
gsr_loss_luma_fwd_bwd = _wrap("gsr_loss_luma_fwd_bwd")

EXPORTED = tuple(_SIGNATURES)
