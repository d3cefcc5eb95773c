"""Moving window along x1 for the oracle (the Sec. 4.1 runs use moving-window
boundaries along x1 and periodic ones along x2).

TEST INFRASTRUCTURE ONLY (imported by tests).  Plain numpy on top of the
oracle's step.

Reading (the paper names the boundary and gives no details): the window moves
along +x1 at c = 1 from `start_step` on.  The periodic x1 box is used as a ring:
whenever c t since the start crosses the next multiple of dx1, the window's
trailing column (physical x1 index `origin`) is cleared -- every E, B and J
component stored at that index set to zero, fresh vacuum -- and the particles
whose cell is that column are removed; the cleared column is the window's new
leading column and `origin` advances by one.  No data moves: window index
i_w = (i - origin) mod n1, window position x_w = (x1 - origin dx1) mod L1.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc


class MovingWindow:
    def __init__(self, grid: orc.Grid, start_step: int = 0):
        self.g = grid
        self.start = int(start_step)
        self.steps = 0
        self.origin = 0
        self.shifts = 0

    def after_step(self, F: orc.Fields, P: orc.Particles | None):
        """Call once after every oracle step: performs the shifts the window owes."""
        self.steps += 1
        if self.steps <= self.start:
            return P
        target = math.floor((self.steps - self.start) * self.g.dt / self.g.dx[0] + 1e-9)
        while self.shifts < target:
            P = self._shift(F, P)
        return P

    def _shift(self, F, P):
        col = self.origin
        for nm in orc.Fields.NAMES:
            getattr(F, nm)[..., col] = 0.0
        if P is not None and P.n:
            keep = np.floor(P.x[0] / self.g.dx[0]).astype(np.int64) != col
            P = orc.Particles([x[keep] for x in P.x], [u[keep] for u in P.u], P.w[keep], P.qm)
        self.origin = (self.origin + 1) % self.g.n[0]
        self.shifts += 1
        return P

    def view(self, a):
        """An array of the grid in window order (x1 index 0 = trailing column)."""
        return np.roll(a, -self.origin, axis=-1)

    def window_x1(self, x1):
        """Particle x1 positions in window coordinates."""
        L1 = self.g.n[0] * self.g.dx[0]
        return np.mod(np.asarray(x1) - self.origin * self.g.dx[0], L1)
