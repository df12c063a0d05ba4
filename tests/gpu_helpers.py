"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same state.

Tolerances (one step from the same state, FP32 device arithmetic vs FP64):
  - neighbour counts: bit-exact, except particles with a candidate pair within
    1e-5 of R (|d - R| < 1e-5), or, metric-free, whose k-th and (k+1)-th
    nearest lie within 1e-5 of each other, which are reported and skipped;
  - orientation: 1e-5 rad, or, where the FP32 condition of arg S is worse, the
    derived bound 5 (n_i + 1) 2^-23 / |S_i| (the error of an FP32 sum of
    n_i + 1 unit vectors divided by its length); such particles are counted;
  - position: 1e-5 L, plus v times the orientation tolerance (streaming uses
    the new orientation), modulo L on periodic axes.
"""
from __future__ import annotations

import numpy as np

import paper_2211_15630_gb300 as A

EPS32 = 2.0 ** -23


def wrap(a):
    return np.mod(a + np.pi, 2 * np.pi) - np.pi


def params(**kw):
    return A.aap_params_default(**kw)


def oracle_model(O, p):
    ns = p.nspecies if p.nspecies > 1 else 0
    sp = {}
    if ns:
        sp = dict(species_n=tuple(p.species_n[:ns]), species_v=tuple(p.species_v[:ns]),
                  species_eta=tuple(p.species_eta[:ns]), species_omega=tuple(p.species_omega[:ns]),
                  species_gamma=tuple(tuple(p.species_gamma[8 * a: 8 * a + ns]) for a in range(ns)))
    if p.weight_len > 0:
        sp["weight_table"] = tuple(p.weight_table[:p.weight_len])
    return O.Model(n=p.n, lx=p.lx, ly=p.ly, r=p.r, v=p.v, eta=p.eta, omega=p.omega,
                   gamma=p.gamma, dt=p.dt, seed=p.seed, model=p.model, order=p.order,
                   weight=p.weight, bx=int(p.bx != 0), by=int(p.by != 0), kn=p.kn, **sp)


def compare_one_step(O, p, h, idx=None, band=1e-5, max_bad_frac=0.0):
    """One GPU step from the handle's current state vs one oracle step.

    Returns a dict of statistics; asserts the tolerances above."""
    n = p.n
    x0, y0, t0 = A.aap_get_state(h, n)
    step = A.aap_observe(h).step
    nb_gpu = A.aap_step_neighbours(h, n)
    x1, y1, t1 = A.aap_get_state(h, n)
    m = oracle_model(O, p)
    if idx is None:
        idx = np.arange(n)
    xo, yo, to, nbo, smag, amb = O.step(m, x0, y0, t0.astype(np.float64), step, idx=idx, band=band)
    g_nb = nb_gpu[idx]
    ok = amb == 0
    nb_bad = np.nonzero(ok & (g_nb != nbo))[0]
    assert nb_bad.size == 0, f"neighbour counts differ at {idx[nb_bad[:10]]}: gpu {g_nb[nb_bad[:10]]} oracle {nbo[nb_bad[:10]]}"
    if p.model == A.AAP_LANGEVIN:
        tol_t = np.full(idx.size, 1e-5)
    else:
        tol_t = np.maximum(1e-5, 5.0 * (nbo + 1) * EPS32 / np.maximum(smag, 1e-30))
    dth = np.abs(wrap(t1[idx].astype(np.float64) - to))
    bad_t = np.nonzero(ok & (dth > tol_t))[0]
    vmax = max(p.species_v[:p.nspecies]) if p.nspecies > 1 else p.v
    disp = vmax * (p.dt if p.model == A.AAP_LANGEVIN else 1.0)
    tol_x = 1e-5 * p.lx + disp * np.minimum(tol_t, 2 * np.pi)
    tol_y = 1e-5 * p.ly + disp * np.minimum(tol_t, 2 * np.pi)
    dx = x1[idx] - xo
    dy = y1[idx] - yo
    if not p.bx:
        dx = np.mod(dx + p.lx / 2, p.lx) - p.lx / 2
    if not p.by:
        dy = np.mod(dy + p.ly / 2, p.ly) - p.ly / 2
    bad_x = np.nonzero(ok & ((np.abs(dx) > tol_x) | (np.abs(dy) > tol_y)))[0]
    nbad = len(set(bad_t.tolist()) | set(bad_x.tolist()))
    assert nbad <= max_bad_frac * idx.size, (
        f"{nbad} particles out of tolerance; worst angle {dth[ok].max() if ok.any() else 0:.3g}, "
        f"first {idx[bad_t[:5]]} dth {dth[bad_t[:5]]} tol {tol_t[bad_t[:5]]}; pos {idx[bad_x[:5]]}")
    return {
        "n": int(idx.size), "near_R": int((~ok).sum()),
        "derived_tol": int((tol_t > 1e-5).sum()),
        "max_dtheta_wellcond": float(dth[ok & (tol_t <= 1e-5)].max(initial=0.0)),
        "max_dpos": float(max(np.abs(dx[ok]).max(initial=0.0), np.abs(dy[ok]).max(initial=0.0))),
    }
