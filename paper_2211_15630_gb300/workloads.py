"""Synthetic workload definitions (parameter sets only, no model arithmetic).

Each function returns aap_params for one of the benchmarked workloads; the
initial states are the library's own seeded uniform isotropic states
(the initial condition of the paper's run-time study, Fig. runtime).
"""
from __future__ import annotations

import math

import numpy as np

from . import AAP_LANGEVIN, AAP_VM, aap_params_default


def vicsek_large(eta: float = 0.45, seed: int = 1, **kw):
    """Standard Vicsek model, N = 2^24, L = 2896 (rho = 2.0004), R = 1, v0 = 0.5, periodic."""
    return aap_params_default(n=1 << 24, lx=2896.0, ly=2896.0, r=1.0, v=0.5, eta=eta, seed=seed,
                              model=AAP_VM, **kw)


def metric_free_vicsek(kn: int = 6, eta: float = 0.45, seed: int = 1, **kw):
    """Metric-free Vicsek model (mfVM), N = 2^24, L = 2896 (rho = 2.0004), k nearest, v0 = 0.5, periodic."""
    return aap_params_default(n=1 << 24, lx=2896.0, ly=2896.0, r=1.0, v=0.5, eta=eta, seed=seed,
                              model=AAP_VM, kn=kn, **kw)


def vicsek_small(eta: float = 0.4, seed: int = 1, **kw):
    """Standard Vicsek model, N = 8192, L = 64 (rho = 2), R = 1, v0 = 0.5, periodic."""
    return aap_params_default(n=8192, lx=64.0, ly=64.0, r=1.0, v=0.5, eta=eta, seed=seed,
                              model=AAP_VM, **kw)


def brownian_walls(seed: int = 1, **kw):
    """Overdamped Langevin alignment, N = 2^20 in 724 x 724 (rho = 2.0004), R = 1,
    v0 = 1, Gamma = 1, D = 0.1 (eta = sqrt(2 D)), dt = 0.01, reflecting walls."""
    return aap_params_default(n=1 << 20, lx=724.0, ly=724.0, r=1.0, v=1.0, eta=math.sqrt(0.2),
                              gamma=1.0, dt=0.01, model=AAP_LANGEVIN, bx=1, by=1, seed=seed, **kw)


def ensemble_replicas(count: int = 256, seed: int = 7, nmin_log2: float = 10.0,
                      nmax_log2: float = 18.0, **kw):
    """Phase-diagram sweep: count Vicsek replicas with N log-uniform in
    [2^nmin, 2^nmax], rho in {0.5, 1, 2, 4}, eta uniform in [0.1, 0.7],
    L = sqrt(N / rho), R = 1, v0 = 0.5, periodic, replica r seeded 1000 + r."""
    g = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(round(2.0 ** g.uniform(nmin_log2, nmax_log2)))
        rho = float(g.choice([0.5, 1.0, 2.0, 4.0]))
        eta = float(g.uniform(0.1, 0.7))
        L = max(math.sqrt(n / rho), 3.0)
        out.append(aap_params_default(n=n, lx=L, ly=L, r=1.0, v=0.5, eta=eta, seed=1000 + r,
                                      model=AAP_VM, **kw))
    return out


def surrogate_training(eta: float, seed: int, **kw):
    """Vicsek N = 524,288, L = 512 (rho = 2) for the coarse-grained surrogate."""
    return aap_params_default(n=524288, lx=512.0, ly=512.0, r=1.0, v=0.5, eta=eta, seed=seed,
                              model=AAP_VM, **kw)
