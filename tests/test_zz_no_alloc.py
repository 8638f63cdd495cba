"""gsr_loss_fwd_bwd_static: the loss entry point for callers that cannot
allocate device memory where they evaluate the loss (for example while a
stream is being captured in the global capture mode, where cudaMalloc is an
error, or inside a host application that owns every allocation).  Its scratch
is a fixed array inside the library, so the caller passes only images and
outputs.  It must give what gsr_loss_fwd_bwd gives, call after call.

This file is named to be collected last: it also checks that the fixed array
works after every other test has used the library in the same process."""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_16728_b300 import _lib as L  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _workspace_loss(x, y, lam, stream):
    C, H, W = x.shape
    sz = ctypes.c_size_t()
    L.gsr_loss_workspace_size(C, H, W, ctypes.byref(sz))
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    d = torch.empty_like(x)
    L.gsr_loss_fwd_bwd(_p(x), _p(y), C, H, W, lam, _p(loss), _p(d), _p(ws), sz.value, stream)
    return loss, d


@pytest.mark.parametrize("shape", [(3, 680, 1200), (3, 37, 53)])
def test_static_scratch_loss_matches_workspace_loss_twice(shape):
    C, H, W = shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((21, 22)):  # two calls in a row, different images
        x = torch.tensor(S.random_image(C, H, W, seed=seed), device="cuda")
        y = torch.tensor(S.random_image(C, H, W, seed=seed + 100), device="cuda")
        ref_loss, ref_d = _workspace_loss(x, y, 0.2, stream)
        loss = torch.full((1,), float("nan"), device="cuda")
        d = torch.full_like(x, float("nan"))
        L.gsr_loss_fwd_bwd_static(_p(x), _p(y), C, H, W, 0.2, _p(loss), _p(d), stream)
        torch.cuda.synchronize()
        assert float(loss.item()) == pytest.approx(float(ref_loss.item()), rel=1e-6), call
        scale = float(ref_d.abs().max())
        assert float((d - ref_d).abs().max()) <= 1e-6 * scale, call


def test_static_scratch_rejects_images_beyond_its_limit():
    rc = L.gsr_loss_fwd_bwd_static.raw(ctypes.c_void_p(16), ctypes.c_void_p(16), 3, 1080, 1920, 0.2,
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == L.GSR_ERR_CAPACITY
    assert b"exceeds the fixed scratch" in L.gsr_last_error()
