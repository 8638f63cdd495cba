"""The learned initialiser on the GPU (tcgen05 MLP) against the FP64 oracle of oracle/mlp.py."""
import numpy as np
import pytest

import oracle
import synthetic as S
from mlp_bounds import EXCEPTION_FRAC, EXCEPTION_MIN, adam_bounds, model_bounds, propagated_bounds
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402
from paper_2311_16728_b300.learned_init import LearnedInit  # noqa: E402


def _levels(seed=3, H=120, W=160):
    img = torch.tensor(S.random_image(3, H, W, seed=seed), device="cuda")
    return gsr.pyramid(img, 3)


def _keypoints(M, W=160, H=120, seed=4):
    rng = np.random.default_rng(seed)
    kp = np.stack([rng.uniform(0, W - 1, M), rng.uniform(0, H - 1, M), rng.uniform(0.5, 5, M),
                   rng.normal(0, 1, M), rng.uniform(-np.pi, np.pi, M)], 1).astype(np.float32)
    return kp


def _np_gather(levels, kp):
    M = kp.shape[0]
    x = np.zeros((M, omlp.K0))
    for m in range(M):
        u, v, d, s, th = kp[m]
        for l, img in enumerate(levels):
            _, Hl, Wl = img.shape
            cx, cy = int(np.rint(np.float32(u) * np.float32(2.0 ** -l))), int(np.rint(np.float32(v) * np.float32(2.0 ** -l)))
            for p in range(256):
                px = min(max(cx - 8 + p % 16, 0), Wl - 1)
                py = min(max(cy - 8 + p // 16, 0), Hl - 1)
                x[m, l * 768 + 3 * p:l * 768 + 3 * p + 3] = img[:, py, px]
        x[m, 2304:2308] = [d, s, np.cos(np.float32(th)), np.sin(np.float32(th))]
    return x


def test_patch_gather_matches_numpy():
    levels = _levels()
    kp = _keypoints(37)
    li = LearnedInit(omlp.init_params(3), 37)
    li.gather(levels, torch.tensor(kp, device="cuda"), transpose=True)
    torch.cuda.synchronize()
    ref = omlp.bf16_round(_np_gather([l.cpu().numpy() for l in levels], kp))
    got = li.x[:37].float().cpu().numpy()
    np.testing.assert_allclose(got[:, :2306], ref[:, :2306], rtol=0, atol=0)
    np.testing.assert_allclose(got[:, 2306:2308], ref[:, 2306:2308], atol=2 ** -7)  # device cos / sin
    assert (li.x[37:].float().abs().max().item() == 0) and torch.equal(li.xT, li.x.t())


def _batch(M, seed=5):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.05, p[k].shape).astype(np.float32)
    x = np.zeros((M, omlp.K0), np.float32)
    x[:, :omlp.K_IN] = rng.uniform(0, 1, (M, omlp.K_IN))
    t = rng.normal(0, 1, (M, omlp.N3)).astype(np.float32)
    t[:, omlp.N_OUT:] = 0
    return p, x, t


def _load(li, x):
    xb = torch.tensor(x, device="cuda").to(torch.bfloat16)
    li.x.zero_()
    li.x[:x.shape[0]] = xb
    li.xT.copy_(li.x.t())


# 100 / 300 rows: short tiles; 20,000: the benchmark's batch, whose 2368-deep
# first layer runs 128 x 128 tiles on the 2-stage ring
@pytest.mark.parametrize("M", [100, 300, 20000])
def test_forward_matches_oracle(M):
    p, x, t = _batch(M)
    li = LearnedInit(p, M)
    _load(li, x)
    y = li.forward()
    torch.cuda.synchronize()
    assert int(li.status.item()) == 0
    fw = omlp.forward(p, x)
    got = y[:M].cpu().numpy()
    err = np.abs(got - fw["y"])
    # the hidden activations are rounded to BF16 on both sides; an FP32/FP64
    # difference can move one of them by an ulp, so bound through |W| |h|
    scale = np.abs(fw["W3"]) @ np.abs(fw["h2"]).T
    assert (err <= 2 ** -7 * scale.T + 1e-4).all(), (err / (scale.T + 1e-9)).max()
    assert np.linalg.norm(err) / np.linalg.norm(fw["y"]) < 1e-3


# 200 rows: short tiles; 2,048 and 20,000: the benchmark's batches (20,000
# runs the 2-stage 128 x 128 forward tiles and the 3-stage split-K weight
# gradient of the first layer)
@pytest.mark.parametrize("M", [200, 2048, 20000])
def test_training_gradients_and_adam_match_oracle(M):
    """One training step (Adam step 5 from seeded moments) against the FP64
    oracle: the loss within 1e-3 relative; every element of the six
    gradients within its bar (tests/mlp_bounds.py: both operands of the
    gradient's own GEMM within two BF16 ulps, plus the FP32 summation bound)
    except at most a few elements per tensor, and those within the envelope
    that carries the operand model through the network (cancelling gated
    gradients of near-dead units); the counts, the normwise error and the
    share of elements within 1e-3 relative printed per tensor; then the fused Adam update of every
    master weight and both moments against oracle.adam on the oracle's
    gradients, within the bound that carries the gradient bound through the
    update."""
    p, x, t = _batch(M, seed=7)
    lr, b1, b2, eps, step = 1e-4, 0.9, 0.999, 1e-8, 5
    f32 = lambda v: float(np.float32(v))  # the kernel receives FP32 hyper-parameters
    fw = omlp.forward(p, x)
    L_ref, dy = omlp.loss_and_dy(fw["y"], t, np.ones(omlp.N3))
    g_ref = omlp.backward(fw, dy)
    bounds = model_bounds(fw, dy, g_ref)
    envelope = propagated_bounds(fw, dy, g_ref)
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    li = LearnedInit(p, M, lr=lr)
    _load(li, x)
    rng = np.random.default_rng(11)
    p0, m0, v0 = {}, {}, {}
    for k in names:
        rms = max(float(np.sqrt(np.mean(g_ref[k] ** 2))), 1e-6)
        shape = li.w.t[k].shape
        # moments 100x the gradient's scale: the update then depends on g
        # only weakly, so the gradient envelope leaves the step's check tight
        m0[k] = rng.normal(0.0, 100.0 * rms, shape).astype(np.float32)
        v0[k] = (rng.uniform(0.5, 2.0, shape) * (100.0 * rms) ** 2).astype(np.float32)
        li.m.t[k].copy_(torch.tensor(m0[k]))
        li.v.t[k].copy_(torch.tensor(v0[k]))
        p0[k] = li.w.t[k].cpu().numpy()
    li.step_count.fill_(step - 1)
    target = torch.zeros(li.mpad, omlp.N3, device="cuda")
    target[:M] = torch.tensor(t, device="cuda")
    li.train_step(target, M)
    torch.cuda.synchronize()
    assert int(li.status.item()) == 0
    L = float(li.loss.item())
    print(f"M {M}: loss {L:.6f} vs {L_ref:.6f} (rel {abs(L - L_ref) / L_ref:.1e})")
    assert L == pytest.approx(L_ref, rel=1e-3)
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in li.gradients().items()}
    for k in names:
        err = np.abs(g[k] - g_ref[k])
        rel = np.linalg.norm(g[k] - g_ref[k]) / max(np.linalg.norm(g_ref[k]), 1e-30)
        within = float(np.mean(err <= np.maximum(1e-3 * np.abs(g_ref[k]), 1e-9)))
        beyond = int((err > bounds[k]).sum())
        print(f"  grad {k}: normwise {rel:.2e}, worst err/bar {float((err / (bounds[k] + 1e-300)).max()):.3f}, "
              f"{beyond} of {err.size} beyond the bar (worst err/envelope "
              f"{float((err / (envelope[k] + 1e-300)).max()):.3f}), {100 * within:.1f} % within 1e-3 relative")
        if not (err <= bounds[k]).all():
            bad = np.argwhere(err > bounds[k])
            for ix in bad[np.argsort(-(err / (bounds[k] + 1e-300))[err > bounds[k]])][:4]:
                ix = tuple(int(v) for v in ix)
                info = f"    {k}{ix}: g {g[k][ix]:.6e} g* {g_ref[k][ix]:.6e} err {err[ix]:.2e} bound {bounds[k][ix]:.2e}"
                if k in ("W2", "W3"):
                    act, prev = ("pre2", "h1") if k == "W2" else (None, "h2")
                    j, c = ix
                    info += f"; |{prev}[:, {c}]| sum {np.abs(fw[prev][:, c]).sum():.3e} nonzero {(fw[prev][:, c] != 0).sum()}"
                    if act:
                        info += f"; rows with {act}[:, {j}] > 0: {(fw[act][:, j] > 0).sum()}"
                print(info)
        assert (err <= envelope[k]).all(), (k, int((err > envelope[k]).sum()))
        assert beyond <= max(EXCEPTION_MIN, EXCEPTION_FRAC * err.size), (k, beyond)
        assert rel < 2e-2, (k, rel)
    for k in names:
        lr_a = np.full(p0[k].shape, f32(lr))
        p1, m1, v1 = oracle.adam(p0[k], g_ref[k], m0[k], v0[k], lr_a, step, f32(b1), f32(b2), f32(eps))
        e_p, e_m, e_v = adam_bounds(p0[k], m0[k], v0[k], g_ref[k], envelope[k], f32(lr), step, f32(b1), f32(b2),
                                    f32(eps))
        w1 = li.w.t[k].cpu().numpy().astype(np.float64)
        gm = li.m.t[k].cpu().numpy().astype(np.float64)
        gv = li.v.t[k].cpu().numpy().astype(np.float64)
        moved = np.abs(p1 - p0[k])
        print(f"  adam {k}: param err / bound {float((np.abs(w1 - p1) / e_p).max()):.3f} (step {moved.mean():.1e}, "
              f"bound {e_p.mean():.1e}, err {np.abs(w1 - p1).mean():.1e} mean), m {float((np.abs(gm - m1) / e_m).max()):.3f}, "
              f"v {float((np.abs(gv - v1) / e_v).max()):.3f}")
        assert e_p.mean() <= 0.05 * moved.mean(), (k, "the step's bound should be a few % of the step")
        assert (np.abs(w1 - p1) <= e_p).all(), k
        assert (np.abs(gm - m1) <= e_m).all(), k
        assert (np.abs(gv - v1) <= e_v).all(), k
    # the step counter advanced and the BF16 copies are the updated masters
    assert int(li.step_count.item()) == step
    assert torch.equal(li.w.h["W1h"], li.w.t["W1"].to(torch.bfloat16))
    assert torch.equal(li.w.h["W3hT"], li.w.t["W3"].t().contiguous().to(torch.bfloat16))


def test_training_reduces_the_loss():
    """Targets from a fixed teacher network are learnable: the loss must fall."""
    M = 256
    p, x, _ = _batch(M, seed=9)
    teacher, _, _ = _batch(M, seed=10)
    t = omlp.forward(teacher, x)["y"].astype(np.float32)
    t[:, omlp.N_OUT:] = 0
    li = LearnedInit(p, M, lr=1e-3)
    _load(li, x)
    target = torch.zeros(li.mpad, omlp.N3, device="cuda")
    target[:M] = torch.tensor(t, device="cuda")
    losses = []
    for _ in range(100):
        li.train_step(target, M)
        losses.append(float(li.loss.item()))
    assert losses[-1] < 0.3 * losses[0], losses[::10]


def test_encode_decode_round_trip():
    p = S.tiny_scene(64, seed=2)
    cam = S.tiny_camera()  # identity pose: every Gaussian is 2-4 m in front
    g = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    # keypoints = projections of the Gaussians themselves, at their depth
    pc = (cam.R @ p.mean_op[:, :3].T.astype(np.float64)).T + cam.t
    kp = np.stack([cam.fx * pc[:, 0] / pc[:, 2] + cam.cx, cam.fy * pc[:, 1] / pc[:, 2] + cam.cy, pc[:, 2],
                   np.zeros(64), np.zeros(64)], 1).astype(np.float32)
    li = LearnedInit(omlp.init_params(1), 64)
    kpt = torch.tensor(kp, device="cuda")
    target = torch.zeros(li.mpad, omlp.N3, device="cuda")
    li.encode_targets(g, torch.arange(64, dtype=torch.int32, device="cuda"), kpt, cam, target)
    li.y.copy_(target)
    out = gsr.Gaussians.zeros(100)
    li.decode(kpt, cam, out, 10)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.mean_op[10:74, :3].cpu().numpy(), p.mean_op[:, :3], atol=2e-5)
    np.testing.assert_allclose(out.mean_op[10:74, 3].cpu().numpy(), p.mean_op[:, 3], atol=1e-6)
    np.testing.assert_allclose(out.logscale[10:74, :3].cpu().numpy(), p.logscale[:, :3], atol=2e-5)
    q = out.quat[10:74].cpu().numpy()
    q0 = p.quat / np.linalg.norm(p.quat, axis=1, keepdims=True)
    assert np.allclose(np.abs((q * q0).sum(1)), 1.0, atol=1e-5)  # same rotation up to sign
    np.testing.assert_allclose(out.sh[:, 10:74].cpu().numpy(), p.sh, atol=1e-6)


def test_residual_encode_decode_round_trip():
    """target = enc(g) - enc(h); decoding target + enc(h) gives g back."""
    p, h = S.tiny_scene(64, seed=2), S.tiny_scene(64, seed=9)
    h.mean_op[:, :3] = p.mean_op[:, :3]  # same centres (the keypoints), other shapes and colours
    cam = S.tiny_camera()
    g = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    gh = gsr.Gaussians.from_arrays(h.mean_op, h.quat, h.logscale, h.sh)
    u, v, z = S.project_points(p.mean_op[:, :3], cam)
    kpt = torch.tensor(np.stack([u, v, z, np.zeros(64), np.zeros(64)], 1).astype(np.float32), device="cuda")
    li = LearnedInit(omlp.init_params(1), 64)
    ids = torch.arange(64, dtype=torch.int32, device="cuda")
    base = torch.zeros(li.mpad, omlp.N3, device="cuda")
    res = torch.zeros(li.mpad, omlp.N3, device="cuda")
    li.encode_targets(gh, ids, kpt, cam, base)
    li.encode_targets(g, ids, kpt, cam, res, base=base)
    li.y.copy_(res)
    out = gsr.Gaussians.zeros(64)
    li.decode(kpt, cam, out, 0, base=base)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.mean_op[:, 3].cpu().numpy(), p.mean_op[:, 3], atol=2e-6)
    np.testing.assert_allclose(out.logscale[:, :3].cpu().numpy(), p.logscale[:, :3], atol=3e-5)
    np.testing.assert_allclose(out.sh.cpu().numpy(), p.sh, atol=2e-6)
    q = out.quat.cpu().numpy()
    q0 = p.quat / np.linalg.norm(p.quat, axis=1, keepdims=True)
    assert np.allclose(np.abs((q * q0).sum(1)), 1.0, atol=1e-5)


def test_learned_init_with_zero_correction_is_the_default():
    """A network whose last layer is zero predicts no correction: the learned
    initialiser then writes the default initialisation."""
    from paper_2311_16728_b300.learned_init import init_weights
    from paper_2311_16728_b300.mapping import densify_default, densify_learned
    p = S.room_scene(20000, seed=3)
    cams = [S.tum_camera(4), S.tum_camera(20)]
    q, offs, kps = S.densify_scene(p, cams, 500, seed=6)
    w = init_weights(3)
    w["W3"][:] = 0.0
    w["b3"][:] = 0.0
    li = LearnedInit(w, 500)
    rng = np.random.default_rng(1)
    keyframes = [(c, torch.tensor(rng.uniform(0, 1, (3, c.height, c.width)).astype(np.float32), device="cuda"))
                 for c in cams]
    kpt = [torch.tensor(k, device="cuda") for k in kps]
    a = gsr.Gaussians.from_arrays(q.mean_op, q.quat, q.logscale, q.sh)
    b = gsr.Gaussians.from_arrays(q.mean_op, q.quat, q.logscale, q.sh)
    densify_default(a, keyframes, kpt, offs)
    densify_learned(li, b, keyframes, kpt, offs)
    torch.cuda.synchronize()
    for x, y in zip(a.tensors(), b.tensors()):
        torch.testing.assert_close(y, x, rtol=0, atol=5e-5)
