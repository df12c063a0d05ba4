"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the tests.

Holds none of the method's arithmetic: only numpy draws of particle states with
the shapes and distributions of the paper's workloads (uniform positions in the
box, isotropic or ordered orientations, Fig. runtime caption and Sec. 4.1).
"""
from __future__ import annotations

import numpy as np


def uniform_state(n: int, lx: float, ly: float, seed: int):
    """Positions uniform in [0,Lx) x [0,Ly), angles uniform in [-pi, pi)."""
    g = np.random.default_rng(seed)
    x = g.uniform(0.0, lx, n)
    y = g.uniform(0.0, ly, n)
    th = g.uniform(-np.pi, np.pi, n)
    return x, y, th


def ordered_state(n: int, lx: float, ly: float, seed: int, theta0: float = 0.3):
    """Uniform positions, every angle equal to theta0 (the ordered state)."""
    x, y, _ = uniform_state(n, lx, ly, seed)
    return x, y, np.full(n, theta0)


def clustered_state(n: int, lx: float, ly: float, seed: int, cx: float, cy: float, w: float):
    """All particles in a w x w square at (cx, cy): a dense cluster (band-like load)."""
    g = np.random.default_rng(seed)
    x = np.mod(cx + g.uniform(-w / 2, w / 2, n), lx)
    y = np.mod(cy + g.uniform(-w / 2, w / 2, n), ly)
    th = g.uniform(-np.pi, np.pi, n)
    return x, y, th


def band_state(n: int, lx: float, ly: float, seed: int, frac: float, width: float):
    """A fraction `frac` of particles in a horizontal band of given width, the rest uniform."""
    g = np.random.default_rng(seed)
    nb = int(frac * n)
    x = g.uniform(0.0, lx, n)
    y = np.concatenate([g.uniform(0.4 * ly, 0.4 * ly + width, nb), g.uniform(0.0, ly, n - nb)])
    th = np.concatenate([g.normal(0.0, 0.3, nb), g.uniform(-np.pi, np.pi, n - nb)])
    th = np.mod(th + np.pi, 2 * np.pi) - np.pi
    return x, np.mod(y, ly), th
