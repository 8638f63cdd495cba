"""Pins of the oracle's densification and pruning (Sec. 3.3.1: split or
clone primitives with large loss gradients, as in 3D Gaussian splatting;
prune nearly transparent ones): the decision table on hand-made cases
including the thresholds themselves, split geometry in closed form for
identity and 90-degree rotations (and an unnormalised quaternion), the
shrunk log-scale, and the covariance of many split children against
R S^2 R^T."""
import numpy as np

import oracle

THR = np.float32(2e-4)
LOGIT_MIN = np.float32(np.log(0.005 / 0.995))
SPLIT = np.float32(np.log(0.05))
SHRINK = np.float32(np.log(1.6))


def _one(mo, q, ls):
    return (np.array([mo], np.float32), np.array([q], np.float32), np.array([list(ls) + [0.0]], np.float32))


def test_decision_table():
    mo = np.array([[0, 0, 3, -6.0],           # A: transparent -> pruned whatever its gradient
                   [0, 0, 3, 0.0],            # B: g == threshold, small -> clone
                   [0, 0, 3, 0.0],            # C: g just below -> keep
                   [0, 0, 3, 0.0],            # D: g above, large -> split
                   [0, 0, 3, 0.0],            # E: never seen -> keep
                   [0, 0, 3, LOGIT_MIN]],     # F: opacity at the bound -> kept (strict <)
                  np.float32)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (6, 1))
    ls = np.tile(np.array([-4.0, -4.0, -4.0, 0.0], np.float32), (6, 1))
    ls[3, 1] = -2.0  # D's largest scale e^-2 > 0.05
    count = np.array([4, 4, 4, 2, 0, 1], np.float32)
    stat = np.array([1.0, 4 * THR, 4 * np.nextafter(THR, np.float32(0)), 1.0, 0.0, 0.0], np.float32)
    eps = np.zeros((6, 6), np.float32)
    out = oracle.densify(mo, q, ls, stat, count, eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    assert out["src"].tolist() == [1, 1, 2, 3, 3, 4, 5]
    assert out["kind"].tolist() == [0, 1, 0, 2, 3, 0, 0]
    # an empty slot (zero quaternion) is dropped even with a large gradient
    q2 = q.copy()
    q2[1] = 0
    out = oracle.densify(mo, q2, ls, stat, count, eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    assert out["src"].tolist() == [2, 3, 3, 4, 5]


def test_split_children_closed_forms():
    s = np.exp(np.float32([-1.0, -2.0, -3.0]).astype(np.float64))
    eps = np.array([[1, 0, 0, 0, 0, -2]], np.float32)
    mo, q, ls = _one([0.5, -0.25, 3.0, 0.0], [1, 0, 0, 0], [-1.0, -2.0, -3.0])
    out = oracle.densify(mo, q, ls, [1.0], [1.0], eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    assert out["kind"].tolist() == [2, 3]
    assert np.allclose(out["mean"][0], [0.5 + s[0], -0.25, 3.0], atol=1e-12)
    assert np.allclose(out["mean"][1], [0.5, -0.25, 3.0 - 2 * s[2]], atol=1e-12)
    shr = np.float32(np.float32([-1.0, -2.0, -3.0]) - SHRINK).astype(np.float64)
    assert np.array_equal(out["logscale"][0], shr) and np.array_equal(out["logscale"][1], shr)
    # 90 degrees about z (unnormalised quaternion): x-axis offsets go along y
    c = np.cos(np.pi / 4)
    mo, q, ls = _one([0.0, 0.0, 3.0, 0.0], [3 * c, 0, 0, 3 * c], [-1.0, -2.0, -3.0])
    out = oracle.densify(mo, q, ls, [1.0], [1.0], np.array([[1, 0, 0, 0, 1, 0]], np.float32), THR, LOGIT_MIN,
                         SPLIT, SHRINK)
    assert np.allclose(out["mean"][0], [0.0, s[0], 3.0], atol=1e-7)
    assert np.allclose(out["mean"][1], [-s[1], 0.0, 3.0], atol=1e-7)


def test_split_children_follow_the_covariance():
    rng = np.random.default_rng(3)
    n = 40000
    q0 = rng.standard_normal(4)
    q0 /= np.linalg.norm(q0)
    ls0 = np.array([-1.0, -1.7, -2.5])
    mo = np.tile(np.array([0, 0, 3, 0], np.float32), (n, 1))
    q = np.tile(q0.astype(np.float32), (n, 1))
    ls = np.tile(np.concatenate([ls0, [0]]).astype(np.float32), (n, 1))
    eps = rng.standard_normal((n, 6)).astype(np.float32)
    out = oracle.densify(mo, q, ls, np.ones(n), np.ones(n), eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    d = out["mean"] - np.array([0, 0, 3.0])
    cov = d.T @ d / len(d)
    w, x, y, z = q0
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    ref = R @ np.diag(np.exp(2 * ls0.astype(np.float32).astype(np.float64))) @ R.T
    assert np.abs(cov - ref).max() <= 0.03 * np.abs(ref).max()
    # and R is a rotation: the sample covariance's eigenvalues are the squared scales
    assert np.allclose(np.sort(np.linalg.eigvalsh(cov)), np.sort(np.exp(2 * ls0)), rtol=0.05)
