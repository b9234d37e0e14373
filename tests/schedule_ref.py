"""Plain restatement of the training routine of Sec. 4.3.2 (delayed start and early
stop of the transform updates) and the plateau scheduler of Sec. 5.2, one brick at
a time, in the readings the library documents (include/srn.h, srn_schedule):

  * the transforms are trained from iteration delay + 1 on;
  * they stop for good once the mean of L_den over the last `window` density
    iterations is not below the mean of the window before by a relative `rel`,
    or once the next iteration would exceed frac * total;
  * L_rec "improves" when it is below the best so far by a relative `prel`; more
    than `pwin` iterations without improvement cut the learning rate by `pfactor`
    and restart the count; the `pmax`-th cut finishes the brick.

Thresholds are taken as the float32 values the library stores."""
import numpy as np


def f32(x):
    return float(np.float32(x))


class BrickRoutine:
    def __init__(self, delay, window, rel, frac, total, pwin, prel, pfactor, pmax):
        self.delay, self.window, self.rel, self.frac, self.total = delay, window, f32(rel), f32(frac), total
        self.pwin, self.prel, self.pfactor, self.pmax = pwin, f32(prel), f32(pfactor), pmax
        self.it = 0
        self.plateaus = 0
        self.bad = 0
        self.finished = False
        self.best = None
        self.den_hist = []
        self.den_stopped = False
        self.den_on = 1 > delay and 1 <= self.frac * total

    def update(self, l_rec, l_den):
        """One iteration's losses (L_den only counts when this iteration trained G)."""
        if not self.finished:
            if self.it == 0 or l_rec < self.best * (1.0 - self.prel):
                self.best, self.bad = l_rec, 0
            else:
                self.bad += 1
            if self.bad > self.pwin:
                self.plateaus += 1
                self.bad = 0
                self.finished = self.plateaus >= self.pmax
            if self.den_on:
                self.den_hist.append(l_den)
                W = self.window
                if len(self.den_hist) >= 2 * W:
                    now = sum(self.den_hist[-W:]) / W
                    before = sum(self.den_hist[-2 * W:-W]) / W
                    if not now < before - self.rel * abs(before):
                        self.den_stopped = True
        self.it += 1
        nxt = self.it + 1
        self.den_on = (not self.finished) and (not self.den_stopped) and nxt > self.delay and nxt <= self.frac * self.total

    @property
    def lr_scale(self):
        return self.pfactor ** self.plateaus
