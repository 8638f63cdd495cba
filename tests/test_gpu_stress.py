"""Stress scene for the backward's transmittance recovery: stacks of large,
nearly opaque Gaussians on the optical axis (opacity up to the 0.99 alpha
clamp), where T_i = T_{i+1} / (1 - alpha_i) divides by numbers down to 0.01.
The gradient bar is the same as for the plain tiny scene: per element
|g - g*| <= max(1e-3 |g*|, 1e-6) against the FP64 oracle, cancellation cases
counted and bounded (parity_helpers.assert_grad_bar); the image within 1e-4
outside flagged pixels."""
import numpy as np
import pytest

import oracle
import synthetic as S
from parity_helpers import (IMG_ATOL, MARGIN_FLAG, assert_grad_bar, colour_clamp_waiver, gpu_view, grad_planes_gpu,
                            oracle_scene, param_condition)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _stack(logit: float, n_stack: int = 24, n_rand: int = 512, seed: int = 0) -> S.Params:
    rng = np.random.default_rng(seed)
    base = S.tiny_scene(n_rand, seed=seed)
    mean = np.stack([rng.normal(0, 0.08, n_stack), rng.normal(0, 0.06, n_stack),
                     2.0 + 0.1 * np.arange(n_stack)], 1)
    op = logit + rng.normal(0, 0.3, n_stack)
    q = rng.standard_normal((n_stack, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ls = np.log(rng.uniform(0.08, 0.2, (n_stack, 3)))
    sh = np.concatenate([rng.uniform(-1, 1, (n_stack, 3)), rng.normal(0, 0.1, (n_stack, 45))], 1)
    mo = np.concatenate([base.mean_op, np.concatenate([mean, op[:, None]], 1)]).astype(np.float32)
    qq = np.concatenate([base.quat, q]).astype(np.float32)
    ll = np.concatenate([base.logscale, np.concatenate([ls, np.zeros((n_stack, 1))], 1)]).astype(np.float32)
    sh_s = np.ascontiguousarray(sh.reshape(n_stack, 12, 4).transpose(1, 0, 2)).astype(np.float32)
    return S.Params(mo, qq, ll, np.concatenate([base.sh, sh_s], 1))


@pytest.mark.parametrize("logit", [2.0, 4.0, 6.0])
def test_stacked_opaque_gaussians(logit):
    p, cam = _stack(logit), S.tiny_camera()
    ca = cam.as_array()
    vb, g = gpu_view(p, cam)
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, cam.width, cam.height)
    sc = oracle_scene(p)
    img, T, nc, mg = oracle.render(sc, ca, cam.width, cam.height, dec)
    flagged = mg < MARGIN_FLAG
    err = np.abs(vb.img.cpu().numpy().astype(np.float64) - img).max(axis=0)
    dimg = S.random_grad_image(3, cam.height, cam.width, seed=3)
    dimg[:, flagged] = 0.0
    gref, g2ref, mag = oracle.render_bwd(sc, ca, cam.width, cam.height, dec, dimg.astype(np.float64),
                                         with_magnitude=True)
    grads = g.zeros_like()
    vb.render_bwd(g, grads, dimg=torch.tensor(dimg, device="cuda"))
    torch.cuda.synchronize()
    pr = oracle.project(sc, ca, cam.width, cam.height, dec.visible)
    clamped = int((pr[:, 5] >= 0.99).sum())
    print(f"logit {logit}: image err {err[~flagged].max():.2e} ({flagged.sum()} flagged); min T "
          f"{T.min():.2e}; Gaussians at the alpha clamp {clamped}")
    assert err[~flagged].max() <= IMG_ATOL
    assert_grad_bar(f"stack logit {logit}, parameter gradients", grad_planes_gpu(grads), gref,
                    param_condition(sc, ca, cam.width, cam.height, dec, mag), waive=colour_clamp_waiver(pr, dec.visible))
