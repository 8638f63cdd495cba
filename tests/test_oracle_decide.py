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
