"""srn_rebalance (host only): after bricks finish, their shares of the batch go to the
bricks still training.  Checked against a plain restatement in exact rational
arithmetic (largest remainder, ties to the lower index) and against its invariants."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2308_02494_gb300 import build as pb
from paper_2308_02494_gb300 import srn


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pb.build()
    srn.load()


def _plain(base, finished, min_points):
    """Proportional shares by largest remainder, in fractions."""
    base = [int(c) for c in base]
    active = [b for b in range(len(base)) if not finished[b]]
    if not active or len(active) == len(base):
        cnt = list(base)
    else:
        cnt = [min(min_points, c) if finished[b] else c for b, c in enumerate(base)]
        freed = sum(base[b] - cnt[b] for b in range(len(base)) if finished[b])
        w = sum(base[b] for b in active)
        share = {b: Fraction(freed * base[b], w) for b in active}
        for b in active:
            cnt[b] += int(share[b])            # floor (non-negative)
        left = freed - sum(int(share[b]) for b in active)
        order = sorted(active, key=lambda b: (-(share[b] - int(share[b])), b))
        for b in order[:left]:
            cnt[b] += 1
    return [0] + list(np.cumsum(cnt, dtype=np.int64).tolist())


def test_matches_the_plain_restatement_on_random_cases():
    r = np.random.default_rng(5)
    for _ in range(400):
        n = int(r.integers(1, 65))
        base = r.integers(1, 1 << int(r.integers(1, 22)), n)
        fin = r.random(n) < r.random()
        mp = int(r.integers(1, 5000))
        got = srn.srn_rebalance(base.tolist(), fin.tolist(), mp)
        assert got == _plain(base, fin, mp)
        cnt = np.diff(got)
        assert got[-1] == int(base.sum())                  # the batch keeps its size
        assert np.all(cnt >= 1)
        if 0 < fin.sum() < n:
            assert np.all(cnt[fin] == np.minimum(mp, base[fin]))
            assert np.all(cnt[~fin] >= base[~fin])
            # every unfinished brick is within one point of its exact proportional share
            freed = int((base[fin] - cnt[fin]).sum())
            exact = base[~fin] + freed * base[~fin] / base[~fin].sum()
            assert np.all(np.abs(cnt[~fin] - exact) < 1.0 + 1e-9)


def test_worked_example_and_degenerate_cases():
    # 580 points freed by bricks 1 and 3 go 1:3 to bricks 0 and 2
    assert srn.srn_rebalance([100, 200, 300, 400], [0, 1, 0, 1], 10) == [0, 245, 255, 990, 1000]
    # nobody finished, everybody finished: the base counts
    assert srn.srn_rebalance([100, 200, 300], [0, 0, 0], 10) == [0, 100, 300, 600]
    assert srn.srn_rebalance([100, 200, 300], [1, 1, 1], 10) == [0, 100, 300, 600]
    # a finished brick smaller than min_points gives nothing up
    assert srn.srn_rebalance([7, 5, 3], [1, 0, 0], 10) == [0, 7, 12, 15]
    # brick 3 frees 2 points: three equal shares of 2/3 floor to 0, and the two points
    # left go to the lower indices
    assert srn.srn_rebalance([1, 1, 1, 3], [0, 0, 0, 1], 1) == [0, 2, 4, 5, 6]
    # srn_read_schedule's dicts work as the finished flags
    assert srn.srn_rebalance([10, 10], [{"finished": 1}, {"finished": 0}], 4) == [0, 4, 20]


def test_large_counts_do_not_overflow():
    big = [(1 << 50) + 3, (1 << 50) - 1, 12345]
    got = srn.srn_rebalance(big, [1, 0, 0], 1)
    assert got == _plain(big, [1, 0, 0], 1)


@pytest.mark.parametrize("args", [
    ([], [], 1),                 # no bricks
    ([5, 0], [0, 0], 1),         # a brick without points
    ([5, 6], [0, 1], 0),         # min_points < 1
    ([1] * 65, [0] * 65, 1),     # more bricks than SRN_MAX_BRICKS
    ([1 << 57], [0], 1),         # beyond the supported range
])
def test_bad_arguments_are_rejected(args):
    with pytest.raises(srn.SrnError) as ei:
        srn.srn_rebalance(*args)
    assert ei.value.status == srn.SRN_ERR_INVALID_ARG
