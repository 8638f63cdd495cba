"""Spatial order of the map store (gsr_spatial_order, gsr_permute): the
permutation is a permutation, sorted by the Morton code of the means (computed
here in integers from the same FP32 quantisation) with equal codes in index
order; permuting moves every plane; the render of a permuted store equals the
render of the original (the image and the per-Gaussian gradients, mapped back,
up to FP32 atomic order)."""
import numpy as np
import pytest

import synthetic as S
from parity_helpers import morton_codes, to_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402


@pytest.mark.parametrize("n", [1, 1000, 70001])
def test_spatial_order_is_the_stable_morton_sort(n):
    p = S.room_scene(n, seed=3)
    # a few means outside the box: clamped to its faces
    if n > 10:
        p.mean_op[:5, 0] = [-9.0, 9.0, -3.0, 3.0, 0.0]
    g = to_gpu(p)
    perm = gsr.spatial_order(g, S.ROOM_LO, S.ROOM_HI).cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(n))
    code = morton_codes(p.mean_op[:, :3], S.ROOM_LO, S.ROOM_HI)
    ref = np.lexsort((np.arange(n), code))  # by code, then index
    assert np.array_equal(perm, ref)


def test_permute_moves_every_plane_and_renders_the_same():
    p = S.perturb(S.room_scene(20000, seed=4), 0.05, seed=5)
    g = to_gpu(p)
    perm = gsr.spatial_order(g, S.ROOM_LO, S.ROOM_HI)
    h = gsr.permuted(g, perm)
    torch.cuda.synchronize()
    pi = perm.long()
    for a, b in zip(g.tensors(), h.tensors()):
        if a.dim() == 3:  # SH planes: (12, n, 4)
            assert torch.equal(b, a[:, pi])
        else:
            assert torch.equal(b, a[pi])
    cam = gsr.camera_from(S.replica_camera(3))
    tiling = gsr.tiling_struct(16, 16)
    out = []
    for store in (g, h):
        vb = gsr.ViewBuffers(store.n, cam, tiling, 1024)
        gsr.ensure_capacity(vb, store)
        vb.forward(store)
        dimg = torch.full_like(vb.img, 1e-3)
        grads = store.zeros_like()
        vb.render_bwd(store, grads, dimg=dimg)
        torch.cuda.synchronize()
        out.append((vb.img.clone(), grads))
    (img0, gr0), (img1, gr1) = out
    # equal depths are the only order the permutation can change; a random
    # scene has none, so the image is the same bit for bit
    assert torch.equal(img0, img1)
    # the gradients are FP32 atomic sums over pixels and tiles in no fixed
    # order (in either store): an element's error scales with the sum of its
    # terms' magnitudes, not with its value, so the bar is normwise plus an
    # absolute one against the plane's largest entry
    for a, b in zip(gr0.tensors(), gr1.tensors()):
        a_p = a[:, pi] if a.dim() == 3 else a[pi]
        scale = float(a.abs().max()) + 1e-30
        assert float((b - a_p).norm()) <= 1e-5 * float(a.norm()) + 1e-30
        assert float((b - a_p).abs().max()) <= 5e-5 * scale
