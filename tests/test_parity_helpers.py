"""Host logic of the gradient bar (parity_helpers.assert_grad_bar and the
colour-clamp waiver), checked on planted errors."""
import numpy as np
import pytest

from parity_helpers import GRAD_TAU, assert_grad_bar, colour_clamp_waiver


def _base(n=400, seed=0):
    rng = np.random.default_rng(seed)
    ref = rng.standard_normal((n, 60))
    cond = 3.0 * np.abs(ref) + 1e-3
    return ref, cond


def test_plain_bar_passes_and_reports():
    ref, cond = _base()
    g = ref * (1 + 5e-4)
    rep = assert_grad_bar("plain", g, ref, cond)
    assert rep["plain"] == rep["checked"] == ref.size and rep["cancellation"] == 0


def test_a_plain_miss_fails():
    ref, cond = _base()
    g = ref.copy()
    g[7, 12] = ref[7, 12] * (1 + 2e-3)  # not a cancellation case: C is 3 |g*|
    with pytest.raises(AssertionError, match="out of tolerance"):
        assert_grad_bar("planted", g, ref, cond)


def test_cancellation_case_is_accepted_and_counted():
    ref, cond = _base()
    ref[3, 40], cond[3, 40] = 1e-9, 1.0  # terms of magnitude ~1 summing to ~0
    g = ref.copy()
    g[3, 40] += 0.5 * GRAD_TAU
    rep = assert_grad_bar("cancel", g, ref, cond)
    assert rep["cancellation"] == 1
    # the same error on a well-conditioned element is not accepted
    ref[3, 40], cond[3, 40] = 1e-2, 1e-2
    with pytest.raises(AssertionError):
        assert_grad_bar("cancel", g, ref, cond)


def test_too_many_cancellation_cases_fail():
    ref, cond = _base(n=100)
    ref[:, 12], cond[:, 12] = 1e-9, 1.0
    g = ref.copy()
    g[:, 12] += 0.5 * GRAD_TAU  # 100 of 6,000 elements: above the 0.1 % cap
    with pytest.raises(AssertionError, match="cancellation cases exceed"):
        assert_grad_bar("many", g, ref, cond)


def test_colour_clamp_waiver_covers_that_channel_and_the_mean_only():
    pr = np.ones((3, 16))
    pr[1, 14] = 5e-5  # Gaussian 1: raw green next to the clamp
    w = colour_clamp_waiver(pr)
    assert not w[0].any() and not w[2].any()
    assert w[1, 0:3].all() and not w[1, 3:12].any()
    sh_cols = np.arange(12, 60)
    assert np.array_equal(w[1, 12:], (sh_cols - 12) % 3 == 1)
    ref, cond = _base(n=3)
    g = ref.copy()
    g[1, 13] += 1.0  # a green SH coefficient: waived
    assert assert_grad_bar("waived", g, ref, cond, waive=w)["waived"] == 3 + 16
    g[1, 4] += 1.0  # the rotation: still checked
    with pytest.raises(AssertionError):
        assert_grad_bar("waived", g, ref, cond, waive=w)
