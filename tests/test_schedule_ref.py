"""Pins of the plain training-routine restatement (tests/schedule_ref.py) against the
paper's description (Sec. 4.3.2 "Delayed start", "Early stopping"; Sec. 5.2 plateau
scheduler) on hand-made loss sequences."""
from schedule_ref import BrickRoutine

PAPER = dict(delay=500, window=1000, rel=1e-4, frac=0.8, total=50000, pwin=500, prel=1e-4, pfactor=0.1, pmax=3)


def test_transforms_frozen_for_the_first_500_iterations():
    r = BrickRoutine(**PAPER)
    on = []
    for i in range(600):
        on.append(r.den_on)              # the decision for iteration i + 1
        r.update(1.0 / (i + 1), 1.0 / (i + 1))   # steadily improving losses
    assert not any(on[:500]) and all(on[500:])


def test_density_stops_when_its_moving_average_stalls():
    r = BrickRoutine(**dict(PAPER, delay=0))
    steps = 0
    while r.den_on:
        r.update(1.0 / (steps + 1), 0.5)      # constant L_den: never 0.01% lower
        steps += 1
    assert steps == 2000                     # two full windows are needed to compare


def test_density_keeps_going_while_its_average_falls():
    r = BrickRoutine(**dict(PAPER, delay=0))
    for i in range(5000):
        r.update(1.0 / (i + 1), 1.0 - 1e-4 * i)   # falls by far more than 0.01% per window
    assert r.den_on and not r.den_stopped


def test_density_stops_at_80_percent_of_training():
    r = BrickRoutine(**dict(PAPER, delay=0, total=1000, window=1000))
    for i in range(1000):
        if not r.den_on:
            break
        r.update(1.0 / (i + 1), -float(i))
    assert r.it == 800                       # iteration 801 would exceed 0.8 * 1000


def test_plateau_cuts_the_learning_rate_and_finishes_the_brick():
    r = BrickRoutine(**PAPER)
    r.update(1.0, 0.0)                       # best = 1.0
    for _ in range(500):
        r.update(1.0, 0.0)                   # 500 iterations without improvement: not yet
    assert r.plateaus == 0
    r.update(1.0, 0.0)                       # the 501st: first cut
    assert r.plateaus == 1 and abs(r.lr_scale - 0.1) < 1e-7
    for _ in range(2 * 501):
        r.update(1.0, 0.0)
    assert r.plateaus == 3 and r.finished and not r.den_on
    it = r.it
    r.update(0.1, 0.0)                       # a finished brick no longer changes its routine
    assert r.plateaus == 3 and r.it == it + 1


def test_an_improvement_of_less_than_the_threshold_does_not_count():
    r = BrickRoutine(**dict(PAPER, pwin=2))
    r.update(1.0, 0.0)
    for _ in range(3):
        r.update(1.0 - 5e-5, 0.0)            # 0.005% better: not an improvement
    assert r.plateaus == 1
