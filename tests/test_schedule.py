"""The plain path's Gaussian-pyramid schedule (Eq. 5, Sec. 3.4): the paper
gives no switch points; the reading is that a keyframe starts at the
coarsest of the three levels and moves one level finer every tau_u / 3 of
its uses, reaching level 0 after tau_u = 30 uses, keyframes taken round
robin (one (keyframe, level) view per iteration).  Host logic only."""
import pytest

from paper_2311_16728_b300.mapping import TAU_U, gp_level


def test_three_levels_tau_30():
    assert TAU_U == 30
    seq = [gp_level(u) for u in range(40)]
    assert seq[:10] == [2] * 10 and seq[10:20] == [1] * 10 and seq[20:] == [0] * 20


@pytest.mark.parametrize("levels,tau,first_zero", [(1, 30, 0), (2, 30, 15), (3, 30, 20), (4, 30, 21), (3, 9, 6)])
def test_level_count_and_tau(levels, tau, first_zero):
    seq = [gp_level(u, levels, tau) for u in range(60)]
    assert seq[0] == levels - 1  # coarsest first
    assert all(a >= b for a, b in zip(seq, seq[1:]))  # never coarser again
    assert all(a - b <= 1 for a, b in zip(seq, seq[1:]))  # one level at a time
    assert seq.index(0) == first_zero and set(seq[first_zero:]) == {0}


def test_round_robin_views():
    """Iteration i trains keyframe i mod K at the level of that keyframe's use count."""
    K, uses, views = 8, [0] * 8, []
    for i in range(8 * 30):
        kf = i % K
        views.append((kf, gp_level(uses[kf])))
        uses[kf] += 1
    assert views[:8] == [(k, 2) for k in range(8)]
    assert views[80:88] == [(k, 1) for k in range(8)]  # the 11th use of every keyframe
    assert views[160:168] == [(k, 0) for k in range(8)]  # the 21st use
    assert sum(1 for _, lvl in views if lvl == 2) == 80
