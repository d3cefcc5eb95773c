"""Moving window along x1 in the oracle (oracle/moving_window.py), CPU.

A window moving at c keeps a luminal pulse: with the proposed solver (no x1
dispersion, Sec. 3.1) the pulse stands still in window coordinates and loses
only its dispersive tails to the cleared trailing columns, where Yee's slower
wavelets slip back and are cut; particles leave exactly when the window's
trailing column passes their cell."""
import numpy as np
import pytest

from oracle import moving_window as mw
from oracle import oracle as orc
from oracle.gen_tables import load as load_table
from paper_2004_03754_gb300 import inputs

DX1, DX2 = inputs.DX1, inputs.DX2


def _pulse_runs(cE, cB, nsteps=400, n=(256, 2), r=0.5):
    dt = r * DX1
    g = orc.Grid(n, (DX1, DX2), dt, cE, cB)
    A = orc.Fields(g)
    orc.laser_load(g, A, a0=1.0, Lenv=6 * np.pi, x_front=150 * DX1)
    e0 = A.e2.copy()
    B = A.copy()
    W = mw.MovingWindow(g)
    for _ in range(nsteps):
        orc.step(g, A, None)          # periodic box
        orc.step(g, B, None)          # the same box seen through the moving window
        W.after_step(B, None)
    assert W.shifts == int(round(nsteps * r))
    lost = max(np.abs(getattr(A, nm) - getattr(B, nm)).max() for nm in ("e2", "b3"))
    drift = np.abs(W.view(B.e2) - e0).max()
    return lost, drift


def test_window_keeps_a_luminal_pulse():
    lost_p, drift_p = _pulse_runs(*load_table(16, 0.5, 0.3))
    lost_y, drift_y = _pulse_runs(np.array([1.0]), np.array([1.0]))
    assert lost_p < 2e-5 and drift_p < 1e-4          # proposed: stands still, keeps its energy
    assert lost_y > 5 * lost_p and drift_y > 100 * drift_p


@pytest.mark.parametrize("r", [0.5, 0.25])
def test_particles_leave_with_the_trailing_column(r):
    n, dt = (64, 2), r * DX1
    g = orc.Grid(n, (DX1, DX2), dt, np.array([1.0]), np.array([1.0]))
    F = orc.Fields(g)
    cols = np.array([0, 3, 7, 12])
    x1 = (cols + 0.3) * DX1
    P = orc.Particles([x1, np.full(cols.size, 0.5 * DX2)], [np.zeros(cols.size)] * 3,
                      np.zeros(cols.size))
    W = mw.MovingWindow(g)
    per_cell = int(round(1 / r))                      # steps per one-cell shift
    alive = []
    for step in range(1, 14 * per_cell + 1):
        orc.step(g, F, P)
        P = W.after_step(F, P)
        alive.append(sorted(np.floor(P.x[0] / DX1).astype(int)))
        # window coordinates of the particles at rest move back one cell per shift
        assert np.allclose(W.window_x1(P.x[0]), P.x[0] - W.shifts * DX1)
    for c in cols:
        gone = (c + 1) * per_cell                     # the shift that clears column c
        assert c in alive[gone - 2] and c not in alive[gone - 1], c
