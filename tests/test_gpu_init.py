"""Default initialisation of new primitives on the GPU against the FP64
oracle: means (back-projection) to FP32 rounding, log-scales within 1e-4
(FP32 coordinates and distances), identity rotation and logit(0.1) exactly
or to one rounding, DC colour to FP32 rounding and the other bands zero."""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402
from paper_2311_16728_b300.learned_init import default_init  # noqa: E402


@pytest.mark.parametrize("n,per_kf", [(20000, 700), (3000, 1), (5000, 0)])
def test_default_init_matches_oracle(n, per_kf):
    p = S.room_scene(n, seed=3)
    cam = S.tum_camera(4)
    [(idx, kp)] = S.held_out_keypoints(p, [cam], per_kf, seed=6)
    M = len(idx)
    # the new primitives occupy the last M slots of the map
    order = np.concatenate([np.setdiff1d(np.arange(n), idx), idx])
    q = S.Params(p.mean_op[order].copy(), p.quat[order].copy(), p.logscale[order].copy(), p.sh[:, order].copy())
    off = n - M
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (3, cam.height, cam.width)).astype(np.float32)
    kp[:, 4] = rng.uniform(-np.pi, np.pi, M)
    g = gsr.Gaussians.from_arrays(q.mean_op, q.quat, q.logscale, q.sh)
    default_init(g, torch.tensor(img, device="cuda"), torch.tensor(kp, device="cuda"), cam, off)
    torch.cuda.synchronize()
    ref = oracle.default_init(img, kp, cam.as_array(), q.mean_op[:, :3].astype(np.float64), off)
    mo = g.mean_op.cpu().numpy()
    np.testing.assert_allclose(mo[off:, :3], ref["mean"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(mo[off:, 3], ref["logit"], rtol=1e-7)
    np.testing.assert_allclose(g.logscale.cpu().numpy()[off:, :3], ref["logscale"], atol=1e-4)
    assert np.all(g.logscale.cpu().numpy()[off:, 3] == 0.0)
    assert np.all(g.quat.cpu().numpy()[off:] == np.array([1, 0, 0, 0], np.float32))
    sh = g.sh.cpu().numpy()[:, off:].transpose(1, 0, 2).reshape(M, 48)
    np.testing.assert_allclose(sh, ref["sh"], rtol=1e-6, atol=1e-6)
    # the rest of the map is untouched
    assert np.array_equal(mo[:off], q.mean_op[:off])
    assert np.array_equal(g.sh.cpu().numpy()[:, :off], q.sh[:, :off])
