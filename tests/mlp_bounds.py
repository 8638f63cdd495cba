"""Element-wise error bounds for the learned initialiser's tensor-core MLP
against its FP64 oracle (test infrastructure; no method arithmetic of the
product lives here).

The GPU and the oracle round the same operands to BF16 at the same places,
so the two sides differ only where an FP32 sum (GEMM accumulation order) and
its FP64 counterpart round to different BF16 neighbours, one BF16 ulp
(2^-8 relative, 8 significant bits) apart, and through what such a
difference moves downstream.  The forward test bounds the output by
2^-7 |W3| |h2|: every operand of the last GEMM within 2^-7 (two BF16 ulps)
of the oracle's.  Two bounds per gradient element:

- `model_bounds`, the bar: the same model for each gradient's own GEMM or
  column sum (2 x 2^-7 |A|^T |B|, 2^-7 for the first layer, whose input is
  the same on both sides), plus the FP32 summation bound gamma_n sum |a b|
  (gamma_n = n u / (1 - n u), u = 2^-24).
- `propagated_bounds`, the envelope: the model carried through the network
  in absolute values -- every BF16 operand (h1, h2, dy, dpre2, dpre1) within
  two BF16 ulps of itself plus what its inputs' bounds allow through the
  product that builds it, ReLU masks that may flip where a pre-activation
  lies within its own band of 0 counted in full.  A gated gradient that is
  itself a cancelling sum (dh2 = dy W3, dh1 = dpre2 W2) gets the bound of
  its inputs rather than two ulps of its value: the case where the bar is
  optimistic (units almost never active).  It is loose (many times the value
  for a typical first-layer element), so it is not the bar.

The test asserts every element within the envelope and at most a few
(EXCEPTION_FRAC of a tensor, at least EXCEPTION_MIN) beyond the bar, and
prints both counts.  `tests/test_mlp_bounds.py` pins the bounds on the CPU
against FP32 / BF16 simulations of the tensor-core arithmetic in permuted
summation orders (`simulate`) and shows that a planted mistake leaves the
envelope.  For the Adam step that follows, `adam_bounds` carries a gradient
bound through the update by the mean value theorem.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
TWO_ULPS = 2.0 ** -7


def gamma(n: int) -> float:
    return n * U32 / (1.0 - n * U32)


def model_bounds(fw: dict, dy: np.ndarray, g_ref: dict) -> dict:
    """The tight per-element bar, built like the forward's 2^-7 |W3| |h2|:
    both operands of each gradient's own GEMM or column sum within two BF16
    ulps of the oracle's (the first layer's input is the same on both
    sides), plus the FP32 summation bound."""
    from oracle import mlp as omlp
    M = dy.shape[0]
    U, s = TWO_ULPS, gamma(M)
    dyb = np.abs(omlp.bf16_round(dy))
    dh2 = omlp.bf16_round(dy) @ fw["W3"]
    dpre2 = dh2 * (fw["pre2"] > 0)
    dh1 = omlp.bf16_round(dpre2) @ fw["W2"]
    dpre1 = dh1 * (fw["pre1"] > 0)
    a2, a1 = np.abs(omlp.bf16_round(dpre2)), np.abs(omlp.bf16_round(dpre1))
    h1, h2, x = np.abs(fw["h1"]), np.abs(fw["h2"]), np.abs(fw["xb"])
    out = {"W3": (2 * U + s) * (dyb.T @ h2), "b3": (U + s) * np.abs(dy).sum(0),
           "W2": (2 * U + s) * (a2.T @ h1), "b2": (U + s) * np.abs(dpre2).sum(0),
           "W1": (U + s) * (a1.T @ x), "b1": (U + s) * np.abs(dpre1).sum(0)}
    for k in out:
        assert out[k].shape == np.shape(g_ref[k]), k
    return out


# an element may miss the model bound only within its propagated bound, and
# for at most this share of a tensor's elements (and at least a handful)
EXCEPTION_FRAC = 1e-3
EXCEPTION_MIN = 8


def propagated_bounds(fw: dict, dy: np.ndarray, g_ref: dict) -> dict:
    """Per-element bounds of the six gradients, from the oracle's forward
    dict (oracle.mlp.forward), dL/dy (oracle.mlp.loss_and_dy) and its
    gradients (oracle.mlp.backward, whose BF16 operands it recomputes).

    Every BF16 operand (activations, dy, dpre2, dpre1) may differ from the
    oracle's by two BF16 ulps of itself; those differences are carried
    linearly through the backward products that build the next operand (so
    a gated gradient that is itself a cancelling sum, dh2 = dy W3 or
    dh1 = dpre2 W2, gets the bound of its inputs, not of its value), and
    into each gradient's own GEMM or column sum, with the FP32 summation
    bound on top.  A ReLU mask can differ where the oracle's pre-activation
    lies within its own rounding band of 0; there the gated gradient counts
    in full, and the activation the oracle has as 0 may be as large as that
    band on the other side."""
    from oracle import mlp as omlp
    M = dy.shape[0]
    K0, H, N3 = fw["W1"].shape[1], fw["W2"].shape[0], fw["W3"].shape[0]
    U = TWO_ULPS
    s = gamma(M)
    h1, h2, x = np.abs(fw["h1"]), np.abs(fw["h2"]), np.abs(fw["xb"])
    aW2, aW3 = np.abs(fw["W2"]), np.abs(fw["W3"])
    # forward: pre-activation bands and the activations' error bounds
    e_pre1 = gamma(K0 + 1) * (x @ np.abs(fw["W1"]).T)
    eh1 = U * h1 + e_pre1 * (np.abs(fw["pre1"]) <= e_pre1)
    e_pre2 = eh1 @ aW2.T + gamma(H + 1) * (h1 @ aW2.T)
    unsure1, unsure2 = np.abs(fw["pre1"]) <= e_pre1, np.abs(fw["pre2"]) <= e_pre2
    eh2 = U * h2 + e_pre2 * unsure2
    e_y = eh2 @ aW3.T + gamma(H + 1) * (h2 @ aW3.T)
    # backward operands and their error bounds
    w_live = (np.abs(dy).sum(0) > 0)[None, :]                 # outputs that carry loss
    edy = ((2.0 / M) * e_y + 4 * U32 * np.abs(dy)) * w_live   # dy = 2 w (y - t) / M in FP32
    dyb = np.abs(omlp.bf16_round(dy))
    edyb = edy + U * dyb
    dh2 = omlp.bf16_round(dy) @ fw["W3"]
    e_dh2 = edyb @ aW3 + gamma(N3) * (dyb @ aW3)
    gate2 = (fw["pre2"] > 0) | unsure2
    dpre2 = dh2 * (fw["pre2"] > 0)
    e2 = e_dh2 * gate2 + np.abs(dh2) * unsure2              # dpre2 (FP32) error, flips in full
    a2 = np.abs(omlp.bf16_round(dpre2))
    e2b = e2 + U * a2                                       # its BF16 operand
    dh1 = omlp.bf16_round(dpre2) @ fw["W2"]
    e_dh1 = e2b @ aW2 + gamma(H) * (a2 @ aW2)
    gate1 = (fw["pre1"] > 0) | unsure1
    dpre1 = dh1 * (fw["pre1"] > 0)
    e1 = e_dh1 * gate1 + np.abs(dh1) * unsure1
    a1 = np.abs(omlp.bf16_round(dpre1))
    e1b = e1 + U * a1
    out = {"W3": edyb.T @ h2 + (dyb + edyb).T @ eh2 + s * (dyb.T @ h2),
           "b3": edy.sum(0) + s * np.abs(dy).sum(0),
           "W2": e2b.T @ h1 + (a2 + e2b).T @ eh1 + s * (a2.T @ h1),
           "b2": e2.sum(0) + s * np.abs(dpre2).sum(0),
           "W1": e1b.T @ x + s * (a1.T @ x),
           "b1": e1.sum(0) + s * np.abs(dpre1).sum(0)}
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
