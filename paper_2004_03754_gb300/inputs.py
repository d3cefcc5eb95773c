"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and lays out grids; it holds none of the
method's arithmetic (no field update, interpolation, push or deposit), so both
the CUDA path and the CPU oracle can be fed from it.

Normalised units (Sec. 2.1): c = m_e = e = 1, k_0 = omega_0 = 1.  The
workloads use 32 cells per laser wavelength along x1, dx2 = dx3 = 4 dx1 and
dt = dx1/2 (the resolution the paper's figures use up to a constant factor).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DEFAULT_SEED = 20040375
DX1 = 2.0 * np.pi / 32.0
DX2 = 4.0 * DX1
DT = 0.5 * DX1


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class ParticleSet:
    x: list          # ndim arrays of positions
    u: list          # 3 arrays, u = gamma*beta
    w: np.ndarray    # deposit weight (charge density carried); 0 = test particle
    qm: float = -1.0

    @property
    def n(self) -> int:
        return int(self.w.size)


def plasma(n, dx, ppc, x1_cells, density, uth, seed=DEFAULT_SEED, charge=-1.0):
    """Uniform plasma of ``ppc`` particles per cell in the cells
    x1_cells[0] <= i < x1_cells[1] (all cells along x2, x3), positions uniform
    within each cell, momenta Gaussian with standard deviation ``uth`` (0 = cold).
    Each particle carries charge density charge*density/ppc."""
    g = rng(seed)
    ndim = len(n)
    lo, hi = x1_cells
    cells = [np.arange(lo, hi)] + [np.arange(m) for m in n[1:]]
    grids = np.meshgrid(*reversed(cells), indexing="ij")          # x1 fastest
    idx = [gr.reshape(-1) for gr in reversed(grids)]
    ncell = idx[0].size
    xs = []
    for d in range(ndim):
        base = np.repeat(idx[d].astype(np.float64), ppc)
        xs.append((base + g.random(ncell * ppc)) * dx[d])
    npart = ncell * ppc
    if uth > 0:
        us = [g.normal(0.0, uth, npart) for _ in range(3)]
    else:
        us = [np.zeros(npart) for _ in range(3)]
    w = np.full(npart, charge * density / ppc)
    return ParticleSet(xs, us, w)


def test_electrons(positions):
    """Test electrons at rest (weight 0: pushed, never deposited)."""
    pos = np.asarray(positions, dtype=np.float64)
    npart = pos.shape[0]
    xs = [pos[:, d].copy() for d in range(pos.shape[1])]
    return ParticleSet(xs, [np.zeros(npart) for _ in range(3)], np.zeros(npart))


def random_particles(n, dx, npart, umax=1.0, seed=DEFAULT_SEED, wscale=0.01):
    """Particles at uniform random positions over the whole box with uniform
    random momenta in [-umax, umax] and random weights (parity tests)."""
    g = rng(seed)
    xs = [g.random(npart) * n[d] * dx[d] for d in range(len(n))]
    us = [g.uniform(-umax, umax, npart) for _ in range(3)]
    w = -wscale * g.random(npart)
    return ParticleSet(xs, us, w)


def random_fields(shape, amp=1.0, seed=DEFAULT_SEED):
    """Nine arrays (E1..E3, B1..B3, J1..J3) of uniform noise in [-amp, amp]."""
    g = rng(seed)
    return [g.uniform(-amp, amp, shape) for _ in range(9)]


def random_coeffs(M, seed=DEFAULT_SEED):
    """Stencil coefficients with a leading 1 and decaying random tails."""
    g = rng(seed)
    cE = g.uniform(-1, 1, M) * 0.3 ** np.arange(M)
    cB = g.uniform(-1, 1, M) * 0.3 ** np.arange(M)
    cE[0] = 1.0 + 0.1 * g.random()
    cB[0] = 1.0 + 0.1 * g.random()
    return cE, cB


def ensemble(nruns=256, seed=DEFAULT_SEED):
    """Grid sizes n1 ~ U{256..2048}, n2 ~ U{64..256} and a0 log-uniform in [10, 1e4]
    for an ensemble of independent vacuum runs."""
    g = rng(seed)
    n1 = g.integers(256, 2049, nruns)
    n2 = g.integers(64, 257, nruns)
    a0 = 10.0 ** g.uniform(1.0, 4.0, nruns)
    return n1, n2, a0
