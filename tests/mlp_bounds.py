"""Element-wise error bounds for the learned initialiser's tensor-core MLP
against its FP64 oracle (test infrastructure; no method arithmetic of the
product lives here).

The GPU and the oracle round the same operands to BF16 at the same places,
so the two sides differ only where an FP32 sum (GEMM accumulation order) and
its FP64 counterpart round to different BF16 neighbours, one BF16 ulp
(2^-8 relative, 8 significant bits) apart, and through what such a
difference moves downstream.  The forward test bounds the output by
2^-7 |W3| |h2|: every operand of the last GEMM within 2^-7 (two BF16 ulps)
of the oracle's.  The gradients get the same kind of bound, built on the
magnitude of each gradient's own GEMM or column sum:

  gW3 = dy^T h2          2 x 2^-7 |dy|^T |h2|          (both operands rounded)
  gW2 = dpre2^T h1       2 x 2^-7 |dpre2|^T |h1|
  gW1 = dpre1^T x        2^-7 |dpre1|^T |x|            (x is the same on both sides)
  gb3, gb2, gb1          2^-7 sum_m |d|                (FP32 column sums)

plus the FP32 summation bound gamma_M sum |a b| (gamma_n = n u / (1 - n u),
u = 2^-24).  A ReLU mask can differ where the oracle's pre-activation lies
within its own bound of 0 (two BF16 ulps of every input of its GEMM, plus
the FP32 summation bound): there the masked gradient may be present on one
side only, so its whole magnitude joins the |d| of the bound, and the
activation the oracle has as 0 may be as large as that bound on the other
side, which joins the |h| of the next layer's weight gradient.  Like the
forward's, this is a model bound (each operand element within two BF16 ulps
of the oracle's), not a worst case over every possible cascade of roundings; `tests/test_mlp_bounds.py` pins it on the CPU against
an FP32 / BF16 simulation of the tensor-core arithmetic and shows that a
planted mistake leaves it.  The model misses one kind of element: sums
over units that are almost never active, or of activations whose FP32
pre-activation cancels to near 0, where another valid summation order moves
the value by far more than two BF16 ulps.  `order_spread` measures that per
element: n simulations of the GPU's arithmetic with independently permuted
summation orders; the test's tolerance is the model bound plus
SPREAD_FACTOR times the largest deviation among them.  For the Adam step
that follows, `adam_bounds` carries a gradient bound through the update by
the mean value theorem.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
TWO_ULPS = 2.0 ** -7


def gamma(n: int) -> float:
    return n * U32 / (1.0 - n * U32)


def gradient_bounds(fw: dict, dy: np.ndarray, g_ref: dict) -> dict:
    """Per-element bounds of the six gradients, from the oracle's forward
    dict (oracle.mlp.forward), dL/dy (oracle.mlp.loss_and_dy) and its
    gradients (oracle.mlp.backward, whose BF16 operands it recomputes)."""
    from oracle import mlp as omlp
    M = dy.shape[0]
    K0, H = fw["W1"].shape[1], fw["W2"].shape[0]
    dyb = np.abs(omlp.bf16_round(dy))
    h1, h2, x = np.abs(fw["h1"]), np.abs(fw["h2"]), np.abs(fw["xb"])
    # pre-activations whose sign the two sides may see differently, and how
    # large the activation the oracle has as 0 can then be on the other side
    e_pre1 = gamma(K0 + 1) * (x @ np.abs(fw["W1"]).T)
    e_pre2 = (2 * TWO_ULPS + gamma(H + 1)) * (h1 @ np.abs(fw["W2"]).T)
    unsure1, unsure2 = np.abs(fw["pre1"]) <= e_pre1, np.abs(fw["pre2"]) <= e_pre2
    h1x, h2x = (1 + TWO_ULPS) * e_pre1 * unsure1, (1 + TWO_ULPS) * e_pre2 * unsure2
    dh2 = omlp.bf16_round(dy) @ fw["W3"]
    dpre2 = dh2 * (fw["pre2"] > 0)
    a2 = np.abs(omlp.bf16_round(dpre2)) + np.abs(dh2) * unsure2
    dh1 = omlp.bf16_round(dpre2) @ fw["W2"]
    dpre1 = dh1 * (fw["pre1"] > 0)
    a1 = np.abs(omlp.bf16_round(dpre1)) + np.abs(dh1) * unsure1
    s = gamma(M)
    out = {"W3": (2 * TWO_ULPS + s) * (dyb.T @ h2) + (1 + TWO_ULPS + s) * (dyb.T @ h2x),
           "W2": (2 * TWO_ULPS + s) * (a2.T @ h1) + (1 + TWO_ULPS + s) * (a2.T @ h1x),
           "W1": (TWO_ULPS + s) * (a1.T @ x),
           "b3": (TWO_ULPS + s) * np.abs(dy).sum(0),
           "b2": (TWO_ULPS + s) * (np.abs(dpre2) + np.abs(dh2) * unsure2).sum(0),
           "b1": (TWO_ULPS + s) * (np.abs(dpre1) + np.abs(dh1) * unsure1).sum(0)}
    for k in out:
        assert out[k].shape == np.shape(g_ref[k]), k
    return out


def _bf(a):
    from oracle import mlp as omlp
    return omlp.bf16_round(a).astype(np.float32)


def simulate(params: dict, x: np.ndarray, t: np.ndarray, weight: np.ndarray, rng=None) -> dict:
    """The MLP's training-step gradients in the GPU's arithmetic on the CPU:
    BF16 operands, FP32 sums (numpy's float32 GEMMs), BF16 roundings of the
    activations and gradients where the GPU makes them, FP32 column sums for
    the biases.  With `rng`, every reduction (the K inputs of layer 1, the
    hidden units of layers 2 and 3 and of the backward products, the M rows
    of the weight gradients and bias sums) runs in an independently permuted
    order: another, equally valid FP32 summation order."""
    f = np.float32
    M, K0 = x.shape
    H, N3 = params["W2"].shape[0], params["W3"].shape[0]
    pk = rng.permutation(K0) if rng is not None else np.arange(K0)
    ph1 = rng.permutation(H) if rng is not None else np.arange(H)
    ph2 = rng.permutation(H) if rng is not None else np.arange(H)
    pn = rng.permutation(N3) if rng is not None else np.arange(N3)
    pm = rng.permutation(M) if rng is not None else np.arange(M)
    xb, W1, W2, W3 = _bf(x), _bf(params["W1"]), _bf(params["W2"]), _bf(params["W3"])
    pre1 = (xb[:, pk] @ W1[:, pk].T).astype(f) + params["b1"]
    h1 = _bf(np.maximum(pre1, 0))
    pre2 = (h1[:, ph1] @ W2[:, ph1].T).astype(f) + params["b2"]
    h2 = _bf(np.maximum(pre2, 0))
    y = (h2[:, ph2] @ W3[:, ph2].T).astype(f) + params["b3"]
    w = np.asarray(weight, f)[None, :]
    dy = (f(2.0) * ((y - t) * w) * (f(1.0) / f(M))).astype(f)
    dyb = _bf(dy)
    g = {"W3": (dyb[pm].T @ h2[pm]).astype(f), "b3": dy[pm].sum(0, dtype=f)}
    dpre2 = (dyb[:, pn] @ W3[pn]).astype(f) * (h2 > 0)
    g["W2"] = (_bf(dpre2)[pm].T @ h1[pm]).astype(f)
    g["b2"] = dpre2[pm].sum(0, dtype=f)
    dpre1 = (_bf(dpre2)[:, ph1] @ W2[ph1]).astype(f) * (h1 > 0)
    g["W1"] = (_bf(dpre1)[pm].T @ xb[pm]).astype(f)
    g["b1"] = dpre1[pm].sum(0, dtype=f)
    return {k: v.astype(np.float64) for k, v in g.items()}


def order_spread(params: dict, x: np.ndarray, t: np.ndarray, weight: np.ndarray, g_ref: dict, n: int = 3,
                 seed: int = 0) -> dict:
    """Per element, the largest deviation from the FP64 oracle among n
    simulations in the GPU's arithmetic with independently permuted summation
    orders: how far a valid FP32 / BF16 evaluation of that element can land
    from the oracle.  It is large exactly where the model bound is optimistic
    (units that are almost never active, pre-activations that cancel to near
    0, ReLU masks that flip), and stays at rounding level elsewhere."""
    rng = np.random.default_rng(seed)
    out = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in g_ref.items()}
    for _ in range(n):
        gs = simulate(params, x, t, weight, rng)
        for k in out:
            out[k] = np.maximum(out[k], np.abs(gs[k] - g_ref[k]))
    return out


# the tolerance of an MLP gradient element: the model bound plus this many
# times the summation-order spread
SPREAD_FACTOR = 4.0


def adam_bounds(p0, m0, v0, g, e_g, lr, t, b1, b2, eps):
    """Bounds on |GPU - oracle| of one Adam step's new parameter, first and
    second moment, given the gradient bound e_g (the oracle's g).  Mean value
    theorem on the update lr m_hat / (sqrt(v_hat) + eps) over the interval
    |g' - g| <= e_g, with sqrt(v_hat) >= sqrt(b2 v0 / bc2) there, plus the
    FP32 rounding of the step (a few ulps of each quantity)."""
    bc1, bc2 = 1.0 - b1 ** t, 1.0 - b2 ** t
    ag = np.abs(g) + e_g
    m = b1 * m0 + (1.0 - b1) * g
    v = b2 * v0 + (1.0 - b2) * g * g
    s_min = np.sqrt(b2 * v0 / bc2)
    am = np.abs(b1 * m0) + (1.0 - b1) * ag
    d_dg = (1.0 - b1) / bc1 / (s_min + eps) + (am / bc1) * ((1.0 - b2) * ag / bc2) / (
        np.maximum(s_min, 1e-300) * (s_min + eps) ** 2)
    step = lr * (np.abs(m) / bc1) / (np.sqrt(v / bc2) + eps)
    e_p = lr * d_dg * e_g + 2.0 * U32 * np.abs(p0) + 16.0 * U32 * (step + lr * d_dg * e_g)
    e_m = (1.0 - b1) * e_g + 3.0 * U32 * (np.abs(m) + (1.0 - b1) * e_g)
    e_v = (1.0 - b2) * (2.0 * np.abs(g) + e_g) * e_g + 4.0 * U32 * (v + (1.0 - b2) * ag * ag)
    return e_p, e_m, e_v
