"""Pins for the learned-initialiser MLP oracle (oracle/mlp.py)."""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_round_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 3.0, 65504.0, 1e-40]]).astype(np.float32)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(a), ref)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1)
    assert mlp.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def _tiny(seed=1, M=6):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.05, p[k].shape).astype(np.float32)
    x = np.zeros((M, mlp.K0), np.float32)
    x[:, :mlp.K_IN] = rng.uniform(0, 1, (M, mlp.K_IN))
    t = rng.normal(0, 1, (M, mlp.N3)).astype(np.float32)
    w = np.ones(mlp.N3)
    return p, x, t, w


def test_forward_matches_explicit_loops():
    p, x, t, w = _tiny(M=2)
    fw = mlp.forward(p, x, round_bf16=False)
    # layer by layer with Python sums over the inputs (no matmul)
    for m in range(2):
        h1 = [max(0.0, sum(float(p["W1"][j, k]) * float(x[m, k]) for k in range(mlp.K0)) + float(p["b1"][j]))
              for j in range(0, mlp.H, 37)]
        np.testing.assert_allclose(fw["h1"][m, ::37], h1, rtol=1e-12, atol=1e-12)
    h2 = np.maximum(fw["h1"] @ p["W2"].astype(np.float64).T + p["b2"], 0)
    y = np.array([[sum(float(p["W3"][j, k]) * h2[m, k] for k in range(mlp.H)) + float(p["b3"][j])
                   for j in range(mlp.N3)] for m in range(2)])
    np.testing.assert_allclose(fw["y"], y, rtol=1e-12, atol=1e-12)


def test_backward_matches_central_differences():
    p, x, t, w = _tiny(M=5)
    p64 = {k: v.astype(np.float64) for k, v in p.items()}

    def L(pp):
        return mlp.loss_and_dy(mlp.forward(pp, x, round_bf16=False)["y"], t, w)[0]

    fw = mlp.forward(p64, x, round_bf16=False)
    assert np.abs(fw["pre1"]).min() > 1e-6 and np.abs(fw["pre2"]).min() > 1e-6  # off the ReLU kinks
    _, dy = mlp.loss_and_dy(fw["y"], t, w)
    g = mlp.backward(fw, dy, round_bf16=False)
    rng = np.random.default_rng(4)
    for name, arr in p64.items():
        idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]
        if name == "W1":
            idx = [(i, min(j, mlp.K_IN - 1)) for i, j in idx]
        if name in ("W3", "b3"):
            idx = [(min(i[0], mlp.N_OUT - 1),) + tuple(i[1:]) for i in idx]
        for ix in idx:
            h = 1e-6 * max(1.0, abs(arr[ix]))
            old = arr[ix]
            arr[ix] = old + h
            lp = L(p64)
            arr[ix] = old - h
            lm = L(p64)
            arr[ix] = old
            assert g[name][ix] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9), (name, ix)


def test_padding_outputs_get_no_gradient():
    p, x, t, w = _tiny(M=3)
    fw = mlp.forward(p, x)
    L, dy = mlp.loss_and_dy(fw["y"], t, w)
    g = mlp.backward(fw, dy)
    assert np.all(dy[:, mlp.N_OUT:] == 0)
    assert np.all(g["W3"][mlp.N_OUT:] == 0) and np.all(g["b3"][mlp.N_OUT:] == 0)
