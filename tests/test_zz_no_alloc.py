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


def _static_loss(x, y, lam, stream):
    C, H, W = x.shape
    loss = torch.full((1,), float("nan"), device="cuda")
    d = torch.full_like(x, float("nan"))
    rc = L.gsr_loss_fwd_bwd_static(_p(x), _p(y), C, H, W, lam, _p(loss), _p(d), stream)
    assert rc == 0
    return loss, d


def test_static_scratch_loss_matches_workspace_loss_call_after_call():
    """Calls in a row on one stream, largest first: a full 3 x 680 x 1200
    frame twice, then one whose image is NaN (it leaves NaN in every map
    entry and partial sum it writes), then a small odd 3 x 37 x 53 image
    twice.  Each finite call must give what gsr_loss_fwd_bwd gives on the
    same images (loss 1e-6 relative, dL/dI 1e-6 of its largest value), so
    nothing a later call reads may come from an earlier, larger one."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    plan = [((3, 680, 1200), 21, False), ((3, 680, 1200), 22, False), ((3, 680, 1200), 23, True),
            ((3, 37, 53), 24, False), ((3, 37, 53), 25, False)]
    for call, ((C, H, W), seed, poison) in enumerate(plan):
        x = torch.tensor(S.random_image(C, H, W, seed=seed), device="cuda")
        y = torch.tensor(S.random_image(C, H, W, seed=seed + 100), device="cuda")
        if poison:
            x.fill_(float("nan"))
            loss, _ = _static_loss(x, y, 0.2, stream)
            torch.cuda.synchronize()
            assert np.isnan(float(loss.item()))
            continue
        ref_loss, ref_d = _workspace_loss(x, y, 0.2, stream)
        loss, d = _static_loss(x, y, 0.2, stream)
        torch.cuda.synchronize()
        rel = abs(float(loss.item()) - float(ref_loss.item())) / abs(float(ref_loss.item()))
        scale = float(ref_d.abs().max())
        derr = float((d - ref_d).abs().max()) / scale
        print(f"call {call} ({C}x{H}x{W}): loss rel diff {rel:.1e}, dL/dI max diff {derr:.1e} of max")
        assert rel <= 1e-6, call
        assert derr <= 1e-6, call


def test_static_scratch_rejects_images_beyond_its_limit():
    rc = L.gsr_loss_fwd_bwd_static.raw(ctypes.c_void_p(16), ctypes.c_void_p(16), 3, 1080, 1920, 0.2,
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == L.GSR_ERR_CAPACITY
    assert b"exceeds the fixed scratch" in L.gsr_last_error()
