"""Camera pose gradient (gsr_pose_bwd) against the FP64 oracle, and a
photometric pose refinement that uses it.

Bars: per element |g - g*| <= max(1e-3 |g*|, 1e-6), with the loss-driven
cases scaled by 3HW (sum-reduced loss); a miss is accepted only as a
cancellation case within 2^-15 C, C the element's condition magnitude (the
oracle's per-Gaussian parts pushed through the absolute value of their
Jacobian in the screen-space gradients, times those gradients' own
condition magnitudes), as for the parameter gradients.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from parity_helpers import MARGIN_FLAG, assert_grad_bar, gpu_view, morton_permuted, oracle_scene, to_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402


def _cam():
    return S.pose_camera((0.1, 0.05, 0.0), 0.05, 150.0, 150.0, 160, 120)


def _pose_condition(sc, ca, W, H, dec, g2mag):
    """sum over Gaussians and screen-space elements k of |d part / d g2_k| * g2mag_k."""
    C = np.zeros(15)
    for k in range(9):
        e = np.zeros((sc.n, 9))
        e[:, k] = g2mag[:, k]
        _, mag = oracle.pose_grad(sc, ca, W, H, dec, e, with_magnitude=True)
        C += mag
    return C


def _gpu_pose(vb, g):
    d = torch.zeros(15, dtype=torch.float32, device="cuda")
    vb.pose_bwd(g, d)
    torch.cuda.synchronize()
    return d.cpu().numpy().astype(np.float64)


def _upload_g2(vb, g2):
    """oracle (N, 9) screen-space gradients -> the device layout (3 planes of float4)."""
    n = g2.shape[0]
    planes = np.zeros((3, n, 4), np.float32)
    planes[0] = g2[:, 0:4]
    planes[1] = g2[:, 4:8]
    planes[2, :, 0] = g2[:, 8]
    vb.g2.copy_(torch.tensor(planes, device="cuda"))


def test_pose_chain_matches_oracle():
    """The chain alone: the oracle's screen-space gradients (FP32-rounded) in."""
    p, cam = S.perturb(S.tiny_scene()), _cam()
    vb, g = gpu_view(p, cam)
    ca = cam.as_array()
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, cam.width, cam.height)
    sc = oracle_scene(p)
    rng = np.random.default_rng(4)
    g2 = rng.standard_normal((p.n, 9)).astype(np.float32).astype(np.float64) * 1e-3
    g2[dec.visible == 0] = 0.0
    _upload_g2(vb, g2)
    got = _gpu_pose(vb, g)
    ref = oracle.pose_grad(sc, ca, cam.width, cam.height, dec, g2)
    cond = _pose_condition(sc, ca, cam.width, cam.height, dec, np.abs(g2))
    print(f"pose chain:\n got {got}\n ref {ref}")
    assert_grad_bar("pose chain, 15 pose values", got[None], ref[None], cond[None])


def test_pose_gradient_end_to_end_matches_oracle():
    """Loss against a frame rendered from the true pose, the camera moved:
    GPU forward, loss, blend backward and pose chain vs the oracle's."""
    base = S.tiny_scene()
    true_cam = _cam()
    tca = true_cam.as_array()
    dec0 = oracle.decide(base.mean_op, base.quat, base.logscale, tca, true_cam.width, true_cam.height)
    gt, _, _, _ = oracle.render(oracle_scene(base), tca, true_cam.width, true_cam.height, dec0)
    cam = S.pose_camera((0.115, 0.04, 0.01), 0.058, 150.0, 150.0, 160, 120)
    ca = cam.as_array()
    dec = oracle.decide(base.mean_op, base.quat, base.logscale, ca, cam.width, cam.height)
    sc = oracle_scene(base)
    img, _, _, mg = oracle.render(sc, ca, cam.width, cam.height, dec)
    L_ref, dimg = oracle.loss(img, gt, 0.2)
    dimg[:, mg < MARGIN_FLAG] = 0.0  # pixels whose FP32 / FP64 decisions may differ
    _, g2ref, mag2d = oracle.render_bwd(sc, ca, cam.width, cam.height, dec, dimg, with_magnitude=True)
    ref = oracle.pose_grad(sc, ca, cam.width, cam.height, dec, g2ref)
    cond = _pose_condition(sc, ca, cam.width, cam.height, dec, mag2d)

    vb, g = gpu_view(base, cam)
    vb.blend_bwd(dimg=torch.tensor(dimg, dtype=torch.float32, device="cuda"))
    got = _gpu_pose(vb, g)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"pose end to end: normwise {rel:.2e}, flagged pixels {(mg < MARGIN_FLAG).sum()}\n got {got}\n ref {ref}")
    # mean-reduced loss: scaled by 3HW (the sum-reduced loss) for the per-element bar
    s = 3 * cam.width * cam.height
    assert_grad_bar("pose end to end (x 3HW), 15 pose values", s * got[None], s * ref[None], s * cond[None])
    assert rel <= 1e-3


def test_pose_gradient_full_size():
    """The pose workload: 300k Gaussians in the Morton-ordered store, 1200 x
    680, target rendered by the oracle from the true pose, camera 1 degree /
    3 cm off; the 15 pose values against the oracle's within the gradient
    bar and 1e-3 normwise."""
    base = morton_permuted(S.room_scene(300_000, seed=0), S.ROOM_LO, S.ROOM_HI)
    true_cam = S.replica_camera(0)
    tca = true_cam.as_array()
    sc = oracle_scene(base)
    dec0 = oracle.decide(base.mean_op, base.quat, base.logscale, tca, true_cam.width, true_cam.height)
    gt, _, _, _ = oracle.render(sc, tca, true_cam.width, true_cam.height, dec0)
    R0 = gsr.so3_exp([0.01, -0.012, 0.006]) @ true_cam.R
    t0 = true_cam.t + np.array([0.02, -0.015, 0.012])
    cam = S.Camera(R0, t0, true_cam.fx, true_cam.fy, true_cam.cx, true_cam.cy, true_cam.width, true_cam.height)
    ca = cam.as_array()
    dec = oracle.decide(base.mean_op, base.quat, base.logscale, ca, cam.width, cam.height)
    img, _, _, mg = oracle.render(sc, ca, cam.width, cam.height, dec)
    _, dimg = oracle.loss(img, gt, 0.2)
    dimg[:, mg < MARGIN_FLAG] = 0.0
    _, g2ref, mag2d = oracle.render_bwd(sc, ca, cam.width, cam.height, dec, dimg, with_magnitude=True)
    ref = oracle.pose_grad(sc, ca, cam.width, cam.height, dec, g2ref)
    cond = _pose_condition(sc, ca, cam.width, cam.height, dec, mag2d)
    vb, g = gpu_view(base, cam)
    vb.blend_bwd(dimg=torch.tensor(dimg, dtype=torch.float32, device="cuda"))
    got = _gpu_pose(vb, g)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"pose full size: normwise {rel:.2e}")
    s = 3 * cam.width * cam.height
    assert_grad_bar("pose full size (x 3HW), 15 pose values", s * got[None], s * ref[None], s * cond[None])
    assert rel <= 1e-3


def test_pose_gradient_is_additive_and_zero_for_zero_screen_gradient():
    p, cam = S.tiny_scene(), _cam()
    vb, g = gpu_view(p, cam)
    vb.g2.zero_()
    assert np.abs(_gpu_pose(vb, g)).max() == 0.0
    rng = np.random.default_rng(5)
    g2 = rng.standard_normal((p.n, 9)) * 1e-3
    _upload_g2(vb, g2)
    d = torch.zeros(15, dtype=torch.float32, device="cuda")
    vb.pose_bwd(g, d)
    once = d.clone()
    vb.pose_bwd(g, d)
    torch.cuda.synchronize()
    # the second pass adds its own sum, whose FP32 atomics may land in another order
    torch.testing.assert_close(d, 2 * once, rtol=1e-5, atol=1e-6 * float(once.abs().max()))


def _angle(R):
    return float(np.arccos(np.clip((np.trace(R) - 1) / 2, -1.0, 1.0)))


def test_pose_refinement_recovers_the_pose():
    """Frame rendered on the GPU from the true pose; refinement from a pose
    1.2 degrees and 2.7 cm away must close most of the gap."""
    p = S.tiny_scene()
    g = to_gpu(p)
    true_cam = _cam()
    vb, _ = gpu_view(p, true_cam)
    gt = vb.img.clone()
    R0 = gsr.so3_exp([0.012, -0.015, 0.008]) @ true_cam.R
    t0 = true_cam.t + np.array([0.02, -0.015, 0.01])
    start = S.Camera(R0, t0, true_cam.fx, true_cam.fy, true_cam.cx, true_cam.cy, true_cam.width, true_cam.height)
    ref = gsr.PoseRefiner(g, start, gt)
    e_rot0, e_t0 = _angle(ref.R @ true_cam.R.T), np.linalg.norm(ref.t - true_cam.t)
    losses = []
    for k in range(200):
        if k == 120:
            ref.lr = ref.lr * 0.1
        losses.append(ref.step())
    e_rot, e_t = _angle(ref.R @ true_cam.R.T), np.linalg.norm(ref.t - true_cam.t)
    print(f"rotation error {np.degrees(e_rot0):.3f} -> {np.degrees(e_rot):.4f} deg; translation "
          f"{e_t0 * 100:.2f} -> {e_t * 100:.3f} cm; loss {losses[0]:.5f} -> {losses[-1]:.6f}")
    assert losses[-1] < 0.2 * losses[0]
    assert e_rot < 0.2 * e_rot0 and e_t < 0.2 * e_t0
