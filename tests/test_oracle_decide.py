"""Pins for the oracle's FP32 decision chain (cull, depth, 3-sigma radius, pixel box) and tile keys.

The chain is an FP32 restatement of the EWA projection cited by Eq. 3; it is
tied here to the oracle's independent FP64 projection, to math.exp, and to a
brute-force pure-Python key builder.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S


def test_chain_exp_close_to_exp():
    xs = np.linspace(-20, 10, 3001, dtype=np.float32)
    for x in xs:
        got = oracle.chain_exp(float(x))
        ref = math.exp(float(x))
        assert abs(got - ref) <= 2 * np.spacing(np.float32(ref)), (x, got, ref)
    assert oracle.chain_exp(0.0) == 1.0


def _scene():
    p = S.tiny_scene(2048, seed=4)
    cam = S.tiny_camera()
    return p, cam, cam.as_array()


def test_decisions_agree_with_fp64_projection():
    p, cam, ca = _scene()
    W, H = cam.width, cam.height
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, W, H)
    sc = oracle.Scene64(p.mean_op, p.quat, p.logscale, p.sh)
    pr = oracle.project(sc, ca, W, H, np.ones(p.n, np.uint8))
    checked = 0
    for i in range(p.n):
        z64 = pr[i, 9]
        assert abs(dec.depth[i] - z64) <= 4 * np.spacing(np.float32(z64))
        if not dec.visible[i]:
            continue
        u, v = pr[i, 0], pr[i, 1]
        assert abs(dec.uv[i, 0] - u) < 1e-4 and abs(dec.uv[i, 1] - v) < 1e-4
        a, b, c = pr[i, 10], pr[i, 11], pr[i, 12]
        mid = 0.5 * (a + c)
        lam = mid + math.sqrt(max(0.1, mid * mid - (a * c - b * b)))
        r3 = 3 * math.sqrt(lam)
        if abs(r3 - round(r3)) < 1e-4:
            continue
        r = math.ceil(r3)
        assert dec.radius[i] == r
        lo_x, hi_x, lo_y, hi_y = u - r, u + r, v - r, v + r
        if min(abs(t - round(t)) for t in (lo_x, hi_x, lo_y, hi_y)) < 1e-4:
            continue
        box = [max(0, math.ceil(lo_x)), min(W - 1, math.floor(hi_x)),
               max(0, math.ceil(lo_y)), min(H - 1, math.floor(hi_y))]
        assert list(dec.box[i]) == box
        checked += 1
    assert checked > 1500


def test_near_plane_and_offscreen_cull():
    cam = S.tiny_camera()
    ca = cam.as_array()
    mean_op = np.array([[0, 0, 0.19, 0], [0, 0, 0.21, 0], [0, 0, -1, 0], [100, 0, 3, 0], [0, 0, 3, 0]], np.float32)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (5, 1))
    ls = np.tile(np.array([-4, -4, -4, 0], np.float32), (5, 1))
    dec = oracle.decide(mean_op, quat, ls, ca, cam.width, cam.height)
    assert list(dec.visible) == [0, 1, 0, 0, 1]


F = np.float32


def _py_tile_keep(u, v, conic, op, x0, x1, y0, y1):
    """The tile cull restated with numpy binary32 scalars (one rounding per op)."""
    A, B, C = (F(c) for c in conic)
    u, v, x0, x1, y0, y1 = F(u), F(v), F(x0), F(x1), F(y0), F(y1)

    def qf(dx, dy):
        return (A * dx * dx + F(2) * B * dx * dy) + C * dy * dy

    if x0 <= u <= x1 and y0 <= v <= y1:
        q = F(0)
    else:
        q = F(np.inf)
        if u < x0 or u > x1:  # the vertical edge facing the mean
            dx = (x0 if u < x0 else x1) - u
            ys = min(max(v - (B * dx) / C, y0), y1)
            q = qf(dx, ys - v)
        if v < y0 or v > y1:  # the horizontal edge facing the mean
            dy = (y0 if v < y0 else y1) - v
            xs = min(max(u - (B * dy) / A, x0), x1)
            q = min(q, qf(xs - u, dy))
    return F(op) * F(oracle.chain_exp(float(F(-0.5) * q))) >= F(0.5) / F(255)


def _edge_min64(u, v, A, B, C, x0, x1, y0, y1, edges):
    """min of the quadratic form over the listed edges of the rectangle, in
    binary64: each edge at its 1D vertex, clamped to the edge."""
    q = np.inf
    for kind, c in edges:
        if kind == "x":
            dx = c - u
            dy = min(max(-B * dx / C, y0 - v), y1 - v)
        else:
            dy = c - v
            dx = min(max(-B * dy / A, x0 - u), x1 - u)
        q = min(q, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    return q


def test_facing_edges_hold_the_rectangle_minimum():
    """The cull's reading: with the mean outside the rectangle, the minimum of
    d^T Q d over it lies on the edges that face the mean.  Checked in binary64
    against all four edges and against a dense sample of the rectangle, over
    random positive-definite forms (elongated and rotated ones included) and
    means in every region around the rectangle."""
    rng = np.random.default_rng(7)
    for _ in range(4000):
        ang, l1 = rng.uniform(0, np.pi), 10 ** rng.uniform(-3, 0)
        l2 = l1 * 10 ** rng.uniform(-3, 0)
        c, s = np.cos(ang), np.sin(ang)
        Q = np.array([[c, -s], [s, c]]) @ np.diag([l1, l2]) @ np.array([[c, s], [-s, c]])
        A, B, C = Q[0, 0], Q[0, 1], Q[1, 1]
        x0, y0 = rng.uniform(0, 50, 2)
        x1, y1 = x0 + rng.uniform(0, 20), y0 + rng.uniform(0, 20)
        u, v = rng.uniform(-40, 110, 2)
        if x0 <= u <= x1 and y0 <= v <= y1:
            continue
        near = ([("x", x0 if u < x0 else x1)] if (u < x0 or u > x1) else []) + \
               ([("y", y0 if v < y0 else y1)] if (v < y0 or v > y1) else [])
        q_near = _edge_min64(u, v, A, B, C, x0, x1, y0, y1, near)
        q_all = _edge_min64(u, v, A, B, C, x0, x1, y0, y1, [("x", x0), ("x", x1), ("y", y0), ("y", y1)])
        assert q_near <= q_all * (1 + 1e-12) + 1e-300, (q_near, q_all)
        xs, ys = np.meshgrid(np.linspace(x0, x1, 17), np.linspace(y0, y1, 17))
        dx, dy = xs - u, ys - v
        assert q_near <= (A * dx * dx + 2 * B * dx * dy + C * dy * dy).min() * (1 + 1e-12)


def _python_keys(dec, W, H, tw, th):
    gx = (W + tw - 1) // tw
    gy = (H + th - 1) // th
    pairs = []
    dbits = dec.depth.view(np.uint32)
    for i in range(len(dec.visible)):
        if not dec.visible[i]:
            continue
        x0, x1, y0, y1 = (int(t) for t in dec.box[i])
        for ty in range(y0 // th, y1 // th + 1):
            for tx in range(x0 // tw, x1 // tw + 1):
                r = (max(tx * tw, x0), min(tx * tw + tw - 1, x1), max(ty * th, y0), min(ty * th + th - 1, y1))
                if _py_tile_keep(dec.uv[i, 0], dec.uv[i, 1], dec.conic[i], dec.opacity[i], *r):
                    pairs.append((((ty * gx + tx) << 32) | int(dbits[i]), i))
    pairs.sort()
    ranges = np.zeros(2 * gx * gy, np.uint32)
    for j, (k, _) in enumerate(pairs):
        t = k >> 32
        if j == 0 or (pairs[j - 1][0] >> 32) != t:
            ranges[2 * t] = j
        ranges[2 * t + 1] = j + 1
    return np.array([k for k, _ in pairs], np.uint64), np.array([g for _, g in pairs], np.uint32), ranges


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 32), (32, 8), (16, 8)])
def test_keys_brute_force(tw, th):
    p, cam, ca = _scene()
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, cam.width, cam.height)
    # force some exact depth ties: they must be ordered by index
    ks, vs, rg = oracle.keys(dec, cam.width, cam.height, tw, th)
    rk, rv, rr = _python_keys(dec, cam.width, cam.height, tw, th)
    assert np.array_equal(ks, rk) and np.array_equal(vs, rv) and np.array_equal(rg, rr)


def test_depth_ties_ordered_by_index():
    cam = S.tiny_camera()
    ca = cam.as_array()
    n = 6
    mean_op = np.zeros((n, 4), np.float32)
    mean_op[:, 2] = 3.0
    mean_op[:, 0] = np.linspace(-0.01, 0.01, n)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    ls = np.tile(np.array([-3, -3, -3, 0], np.float32), (n, 1))
    dec = oracle.decide(mean_op, quat, ls, ca, cam.width, cam.height)
    ks, vs, rg = oracle.keys(dec, cam.width, cam.height)
    for t in range(len(rg) // 2):
        seg = vs[rg[2 * t]:rg[2 * t + 1]]
        assert list(seg) == sorted(seg)


def test_chain_conic_and_opacity_match_fp64():
    p, cam, ca = _scene()
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, cam.width, cam.height)
    sc = oracle.Scene64(p.mean_op, p.quat, p.logscale, p.sh)
    pr = oracle.project(sc, ca, cam.width, cam.height, dec.visible)
    v = dec.visible > 0
    np.testing.assert_allclose(dec.conic[v], pr[v, 2:5], rtol=1e-4, atol=1e-6 * np.abs(pr[v, 2:5]).max())
    np.testing.assert_allclose(dec.opacity[v], pr[v, 5], rtol=1e-6)


def test_dropped_tiles_never_reach_the_alpha_threshold():
    """Every pixel of a dropped (Gaussian, tile) pair has FP64 alpha < 1/255 by a
    wide margin: the cull cannot change the image (so the image stays
    independent of the tile shape)."""
    p, cam, ca = _scene()
    W, H = cam.width, cam.height
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, W, H)
    sc = oracle.Scene64(p.mean_op, p.quat, p.logscale, p.sh)
    pr = oracle.project(sc, ca, W, H, dec.visible)
    dropped = kept = 0
    worst = 0.0
    for tw, th in [(16, 16), (8, 32)]:
        for i in np.flatnonzero(dec.visible):
            x0, x1, y0, y1 = (int(t) for t in dec.box[i])
            u, v, A, B, C, op = pr[i, :6]
            for ty in range(y0 // th, y1 // th + 1):
                for tx in range(x0 // tw, x1 // tw + 1):
                    r = (max(tx * tw, x0), min(tx * tw + tw - 1, x1), max(ty * th, y0), min(ty * th + th - 1, y1))
                    if oracle.tile_keep(dec.uv[i, 0], dec.uv[i, 1], dec.conic[i], dec.opacity[i], *r):
                        kept += 1
                        continue
                    dropped += 1
                    xs, ys = np.meshgrid(np.arange(r[0], r[1] + 1), np.arange(r[2], r[3] + 1))
                    dx, dy = xs - u, ys - v
                    a = op * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
                    worst = max(worst, float(a.max()) * 255)
    assert dropped > 0 and kept > 0
    assert worst < 0.51, worst  # max alpha of any dropped pixel, in units of 1/255
