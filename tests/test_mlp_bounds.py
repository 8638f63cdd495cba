"""CPU pins of the MLP parity bounds (tests/mlp_bounds.py): FP32 / BF16
simulations of the tensor-core arithmetic (BF16 operands, FP32 sums in
other orders, BF16 roundings of activations and gradients at the GPU's
places) stay inside the per-element bounds; their normwise error is far
below them; and a simulation with a planted mistake leaves them."""
import numpy as np

from mlp_bounds import EXCEPTION_FRAC, EXCEPTION_MIN, adam_bounds, model_bounds, propagated_bounds
from oracle import mlp as omlp


def _case(M=96, seed=2):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.05, p[k].shape).astype(np.float32)
    x = np.zeros((M, omlp.K0), np.float32)
    x[:, :omlp.K_IN] = rng.uniform(0, 1, (M, omlp.K_IN))
    t = rng.normal(0, 1, (M, omlp.N3)).astype(np.float32)
    t[:, omlp.N_OUT:] = 0
    return p, x, t


def _bf(a):
    return omlp.bf16_round(a).astype(np.float32)


def _simulate(p, x, t, w, drop_mask=False):
    """FP32 sums of BF16 operands (numpy's float32 GEMM: its own blocking and
    order), BF16 roundings where the GPU makes them."""
    f = np.float32
    xb, W1, W2, W3 = _bf(x), _bf(p["W1"]), _bf(p["W2"]), _bf(p["W3"])
    pre1 = (xb @ W1.T).astype(f) + p["b1"]
    h1 = _bf(np.maximum(pre1, 0))
    pre2 = (h1 @ W2.T).astype(f) + p["b2"]
    h2 = _bf(np.maximum(pre2, 0))
    y = (h2 @ W3.T).astype(f) + p["b3"]
    M = x.shape[0]
    d = (y - t) * w[None, :].astype(f)
    dy = (f(2.0) * d * (f(1.0) / f(M))).astype(f)
    dyb = _bf(dy)
    g = {"W3": (dyb.T @ h2).astype(f), "b3": dy.sum(0, dtype=f)}
    dh2 = (dyb @ W3).astype(f)
    dpre2 = dh2 if drop_mask else dh2 * (h2 > 0)
    g["W2"] = (_bf(dpre2).T @ h1).astype(f)
    g["b2"] = dpre2.sum(0, dtype=f)
    dh1 = (_bf(dpre2) @ W2).astype(f)
    dpre1 = dh1 * (h1 > 0)
    g["W1"] = (_bf(dpre1).T @ xb).astype(f)
    g["b1"] = dpre1.sum(0, dtype=f)
    return y, g


def _setup(seed, M):
    p, x, t = _case(M=M, seed=seed)
    w = np.ones(omlp.N3)
    w[omlp.N_OUT:] = 0
    fw = omlp.forward(p, x)
    _, dy = omlp.loss_and_dy(fw["y"], t, w)
    g_ref = omlp.backward(fw, dy)
    return p, x, t, w, fw, g_ref, (model_bounds(fw, dy, g_ref), propagated_bounds(fw, dy, g_ref))


def _check(g, g_ref, bb, label):
    """Every element within the envelope, at most a few beyond the bar."""
    model, env = bb
    for k in g_ref:
        err = np.abs(g[k] - g_ref[k])
        assert (err <= env[k]).all(), (label, k, float((err / (env[k] + 1e-300)).max()))
        assert int((err > model[k]).sum()) <= max(EXCEPTION_MIN, EXCEPTION_FRAC * err.size), (label, k)


def test_fp32_simulation_inside_the_bounds():
    for seed, M in ((2, 96), (5, 640)):
        p, x, t, w, fw, g_ref, bb = _setup(seed, M)
        y, g = _simulate(p, x, t, w)
        scale = np.abs(fw["W3"]) @ np.abs(fw["h2"]).T
        assert (np.abs(y - fw["y"]) <= 2 ** -7 * scale.T + 1e-4).all()  # the forward test's bound
        _check(g, g_ref, bb, (seed, M))
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            # the actual error sits well inside the bar: normwise below a tenth of its norm
            assert np.linalg.norm(np.abs(g[k] - g_ref[k])) <= 0.1 * np.linalg.norm(bb[0][k]), k


def test_bounds_cover_simulations_in_permuted_orders():
    """Simulations of the GPU's arithmetic whose every reduction runs in an
    independently permuted order (other valid FP32 summation orders, so other
    BF16 roundings downstream) all stay inside the envelope with at most a
    few elements beyond the bar, also at a batch of 2,048 rows with
    near-dead units."""
    from mlp_bounds import simulate
    for seed, M in ((6, 640), (7, 2048)):
        p, x, t, w, fw, g_ref, bb = _setup(seed, M)
        for r in range(3):
            _check(simulate(p, x, t, w, np.random.default_rng(100 + r)), g_ref, bb, (M, r))


def test_planted_mistake_leaves_the_bounds():
    p, x, t, w, fw, g_ref, bb = _setup(4, 96)
    _, g = _simulate(p, x, t, w, drop_mask=True)  # the layer-2 ReLU mask forgotten
    assert (np.abs(g["W2"] - g_ref["W2"]) > bb[1]["W2"]).any()
    assert (np.abs(g["b2"] - g_ref["b2"]) > bb[1]["b2"]).any()


def test_adam_bound_covers_a_perturbed_gradient():
    """An FP32 Adam step on a gradient moved anywhere within its bound lands
    within the step's bound of the FP64 step on the exact gradient."""
    rng = np.random.default_rng(3)
    n = 5000
    g = rng.normal(0, 1e-3, n)
    e_g = np.abs(g) * 1e-2 + 1e-6
    p0 = rng.normal(0, 0.05, n).astype(np.float32)
    m0 = (rng.normal(0, 1e-3, n)).astype(np.float32)
    v0 = (rng.uniform(0.5, 2.0, n) * 1e-6).astype(np.float32)
    lr, t, b1, b2, eps = 1e-3, 5, 0.9, 0.999, 1e-8
    bc1, bc2 = 1 - b1 ** t, 1 - b2 ** t
    m = b1 * m0 + (1 - b1) * g
    v = b2 * v0 + (1 - b2) * g * g
    p1 = p0 - lr * (m / bc1) / (np.sqrt(v / bc2) + eps)
    gp = (g + e_g * rng.uniform(-1, 1, n)).astype(np.float32)
    f = np.float32
    m32 = f(b1) * m0 + f(1 - b1) * gp
    v32 = f(b2) * v0 + f(1 - b2) * gp * gp
    p32 = p0 - f(lr) * (m32 / f(bc1)) / (np.sqrt(v32 / f(bc2)) + f(eps))
    e_p, e_m, e_v = adam_bounds(p0, m0, v0, g, e_g, lr, t, b1, b2, eps)
    assert (np.abs(p32 - p1) <= e_p).all()
    assert (np.abs(m32 - m) <= e_m).all()
    assert (np.abs(v32 - v) <= e_v).all()
