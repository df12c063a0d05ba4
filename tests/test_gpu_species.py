"""Particle species (Sec. 2.5): per-species v, eta, omega and a coupling
matrix Gamma_ab, CUDA path through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from tests.gpu_helpers import compare_one_step, params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _three(**kw):
    base = dict(n=9000, lx=70.0, ly=64.0, seed=41)
    base.update(kw)
    p = params(**base)
    return A.set_species(p, (2000, 3000, 4000), v=(0.2, 0.5, 0.9), eta=(0.1, 0.4, 0.7),
                         omega=(0.0, 0.2, -0.3),
                         gamma=((1.0, 0.5, 0.0), (2.0, 1.0, -0.5), (0.3, 0.0, 1.5)))


@pytest.mark.parametrize("kw", [
    dict(),                                                  # VM
    dict(model=A.AAP_NVM, bx=1),                             # NVM, reflecting in x
    dict(model=A.AAP_LANGEVIN, dt=0.1),                      # Langevin, Gamma matrix, h = 1/(1+n)
    dict(model=A.AAP_LANGEVIN, dt=0.1, order=2, weight=A.AAP_H_ONE, by=1),
    dict(kn=7),                                              # mfVM mixture
    dict(kn=5, model=A.AAP_LANGEVIN, dt=0.1, bx=1, by=1),    # mfL with Gamma matrix
])
def test_species_one_step_matches_oracle(lib, oracle, kw):
    p = _three(**kw)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        compare_one_step(oracle, p, h)
    finally:
        A.aap_destroy(h)


def test_species_in_ensemble_equal_standalone(lib):
    """Replicas with species run batched are bit-identical to standalone runs."""
    ps = [_three(seed=50 + r, model=A.AAP_LANGEVIN, dt=0.05) for r in range(3)]
    ps[1].n = 5000
    A.set_species(ps[1], (4000, 1000), v=(0.3, 0.6), gamma=((0.5, 2.0), (1.0, 0.0)))
    e = A.aap_ens_create(ps)
    try:
        A.aap_ens_step(e, 40)
        for r, p in enumerate(ps):
            lay = A.aap_ens_get_layout(e, r)
            q = A.aap_params_default()
            for f, _ in A.aap_params._fields_:
                setattr(q, f, getattr(p, f))
            q.tile_w, q.tile_h = lay.tile_w, lay.tile_h
            h = A.aap_create(q)
            try:
                A.aap_step(h, 40)
                for u, v in zip(A.aap_ens_get_state(e, r, p.n), A.aap_get_state(h, p.n)):
                    assert np.array_equal(u, v)
            finally:
                A.aap_destroy(h)
    finally:
        A.aap_ens_destroy(e)


def test_single_species_list_equals_scalars(lib):
    """nspecies = 1 is the scalar model, bit for bit."""
    p0 = params(n=20000, lx=100.0, ly=100.0, seed=3, model=A.AAP_LANGEVIN, dt=0.1)
    p1 = params(n=20000, lx=100.0, ly=100.0, seed=3, model=A.AAP_LANGEVIN, dt=0.1)
    A.set_species(p1, (20000,))
    h0, h1 = A.aap_create(p0), A.aap_create(p1)
    try:
        A.aap_step(h0, 10)
        A.aap_step(h1, 10)
        for u, v in zip(A.aap_get_state(h0, p0.n), A.aap_get_state(h1, p1.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h0)
        A.aap_destroy(h1)


def test_weight_table_matches_oracle_and_builtin(lib, oracle):
    """Tabulated Langevin weight h(n) (Sec. 4): one step against the oracle with
    a table shorter than the neighbour numbers (its last entry is reused), and
    an all-ones table equal to h = 1 bit for bit."""
    p = params(n=12000, lx=80.0, ly=80.0, seed=19, model=A.AAP_LANGEVIN, dt=0.1, gamma=2.0)
    A.set_weight_table(p, (0.9, 0.5, 0.45, 0.3, 0.22, 0.2, 0.17))
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        compare_one_step(oracle, p, h)
    finally:
        A.aap_destroy(h)
    p1 = params(n=12000, lx=80.0, ly=80.0, seed=19, model=A.AAP_LANGEVIN, dt=0.1, gamma=2.0,
                weight=A.AAP_H_ONE)
    p2 = params(n=12000, lx=80.0, ly=80.0, seed=19, model=A.AAP_LANGEVIN, dt=0.1, gamma=2.0)
    A.set_weight_table(p2, (1.0, 1.0))
    h1, h2 = A.aap_create(p1), A.aap_create(p2)
    try:
        A.aap_step(h1, 8)
        A.aap_step(h2, 8)
        for u, v in zip(A.aap_get_state(h1, p1.n), A.aap_get_state(h2, p2.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)
