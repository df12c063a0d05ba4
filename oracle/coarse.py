"""FP64 CPU oracle of the coarse-grained fields (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  Parity: pinned by tests/test_coarse_oracle.py (a
hand-worked fixture, conservation of the particle number and of the sum of
e^{i theta}, bin-by-bin interval counting, translation by one bin).

The fields are the density and the polarisation of a state averaged over a
regular grid of nbx x nby bins covering the box [0, lx] x [0, ly]:

    rho(b) = |{i : i in bin b}| / A,      p(b) = sum_{i in b} (cos th_i, sin th_i) / A

with A = (lx / nbx)(ly / nby) the bin area.  Summed over all bins,
A sum_b p(b) = sum_i e^{i theta_i}, so the polar order parameter of the
fields equals the particles' |sum_i e^{i theta_i}| / N (Sec. 3.4).  The paper
defines no such fields; they are what the learned surrogate advances.

A particle's bin along x is floor(x (nbx / lx)) in FP64, the product of the
FP64 position and the FP64 ratio nbx / lx, clamped to [0, nbx) (a position
x = lx belongs to the last bin); the same along y.  Both sides of a
comparison take this integer decision in FP64 from the same FP64 position.
"""
from __future__ import annotations

import numpy as np


def bin_index(u, nb: int, length: float) -> np.ndarray:
    """floor(u (nb / length)) in FP64, clamped to [0, nb - 1]."""
    f = float(nb) / float(length)
    t = np.floor(np.asarray(u, np.float64) * f)
    return np.clip(t, 0, nb - 1).astype(np.int64)


def coarse_grain(x, y, th, lx: float, ly: float, nbx: int, nby: int) -> np.ndarray:
    """Fields [3, nby, nbx]: density, polarisation x, polarisation y per unit
    area (planes row-major with x fastest), from FP64 positions and angles."""
    ix = bin_index(x, nbx, lx)
    iy = bin_index(y, nby, ly)
    th = np.asarray(th, np.float64)
    out = np.zeros((3, nby, nbx))
    np.add.at(out[0], (iy, ix), 1.0)
    np.add.at(out[1], (iy, ix), np.cos(th))
    np.add.at(out[2], (iy, ix), np.sin(th))
    area = (lx / nbx) * (ly / nby)
    return out / area


def counts(x, y, lx: float, ly: float, nbx: int, nby: int) -> np.ndarray:
    """Particle count per bin [nby, nbx] (the density times the bin area)."""
    ix = bin_index(x, nbx, lx)
    iy = bin_index(y, nby, ly)
    c = np.zeros((nby, nbx), np.int64)
    np.add.at(c, (iy, ix), 1)
    return c
