"""Metric-free neighbourhoods (mfVM, mfNVM, mfL; Sec. 2.3): the CUDA path
through the C ABI against the FP64 oracle's brute-force k-nearest search,
one step from the same state (tolerances in tests/gpu_helpers.py)."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from tests import inputs
from tests.gpu_helpers import compare_one_step, params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _mf(**kw):
    base = dict(n=6000, lx=60.0, ly=55.0, v=0.4, eta=0.35, seed=31, kn=6)
    base.update(kw)
    return params(**base)


@pytest.mark.parametrize("kw", [
    dict(),                                              # mfVM, periodic, k = 6
    dict(kn=1), dict(kn=13), dict(kn=32),                # the three register lists
    dict(model=A.AAP_NVM),                               # mfNVM
    dict(model=A.AAP_LANGEVIN, dt=0.1, v=1.0, gamma=1.5),  # mfL (h = 1)
    dict(model=A.AAP_LANGEVIN, dt=0.1, v=1.0, order=2, kn=9),
    dict(bx=1), dict(by=1), dict(bx=1, by=1, kn=10),     # reflecting walls, own images
    dict(bx=1, by=1, model=A.AAP_LANGEVIN, dt=0.05, order=3),
    dict(omega=0.3, lx=90.0, ly=30.0),                   # chirality, elongated box
])
def test_mf_one_step_matches_oracle(lib, oracle, kw):
    p = _mf(**kw)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        st = compare_one_step(oracle, p, h)
        assert st["near_R"] < 0.01 * p.n
    finally:
        A.aap_destroy(h)


def test_mf_clustered_state_expands_rings(lib, oracle):
    """A dense cluster in a mostly empty box: particles at its rim and the few
    outside need many rings (and the exact fallback near half the box)."""
    p = _mf(n=4000, lx=80.0, ly=80.0, kn=7)
    h = A.aap_create(p)
    try:
        x, y, th = inputs.clustered_state(p.n, p.lx, p.ly, 5, 20.0, 30.0, 6.0)
        x[:20] = np.linspace(50.0, 75.0, 20)          # a few strays far from it
        y[:20] = np.linspace(60.0, 10.0, 20)
        A.aap_set_state(h, x, y, th.astype(np.float32), step=0)
        compare_one_step(oracle, p, h)
    finally:
        A.aap_destroy(h)


@pytest.mark.parametrize("n,k,bx,by", [(5, 8, 0, 0), (1, 3, 0, 0), (3, 6, 1, 1), (9, 4, 0, 1), (2, 1, 0, 0)])
def test_mf_tiny_systems(lib, oracle, n, k, bx, by):
    """Fewer candidates than k, a single particle, own mirror images: the
    periodic window cannot certify the list and the exact scan takes over."""
    p = _mf(n=n, lx=7.0, ly=6.0, kn=k, bx=bx, by=by, v=0.3)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 2)
        compare_one_step(oracle, p, h)
    finally:
        A.aap_destroy(h)


def test_mf_deterministic_and_graph_replay(lib):
    """Same parameters, same trajectory bit for bit, whether the 64 steps run
    as captured graphs or one launch at a time (the selected set is ordered by
    distance, id and image, not by arrival in a cell)."""
    p = _mf(n=20000, lx=100.0, ly=100.0, kn=7, model=A.AAP_NVM)
    h1, h2 = A.aap_create(p), A.aap_create(p)
    try:
        A.aap_step(h1, 64)
        for _ in range(64):
            A.aap_step(h2, 1)
        for u, v in zip(A.aap_get_state(h1, p.n), A.aap_get_state(h2, p.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_mf_full_size_sampled(lib, oracle):
    """N = 2^22 at density 2, k = 6: sampled particles against the oracle's
    exact search over all N."""
    p = _mf(n=1 << 22, lx=1448.0, ly=1448.0, kn=6, eta=0.45, v=0.5)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        idx = np.random.default_rng(4).choice(p.n, 200, replace=False)
        compare_one_step(oracle, p, h, idx=np.sort(idx))
    finally:
        A.aap_destroy(h)


def test_mf_measurement_neighbour_number_is_k(lib):
    """|Omega_i| = k for every particle (Sec. 2.3): the mean neighbour number is
    k and the neighbour histogram is a single bin."""
    p = _mf(n=10000, lx=70.0, ly=70.0, kn=5)
    p.binnum_neighbors = 8
    h = A.aap_create(p)
    try:
        A.aap_step(h, 4)
        A.aap_measure(h, 6)
        res = A.aap_get_results(h)
        th_h, nb_h = A.aap_get_histograms(h, 100, 8)
        assert res.samples == 6 and res.nbar[0] == 5.0 and res.nbar[1] == 25.0
        assert nb_h[5] == 1.0 and abs(th_h.sum() - 1) < 1e-12
        obs = A.aap_observe(h)
        assert obs.mean_neighbours == 5.0
    finally:
        A.aap_destroy(h)


def test_mf_save_load_and_ensemble_rejected(lib, tmp_path):
    p = _mf(n=8000, lx=64.0, ly=64.0, kn=6, model=A.AAP_LANGEVIN, dt=0.1, v=1.0)
    h = A.aap_create(p)
    path = str(tmp_path / "mf.aap")
    try:
        A.aap_step(h, 5)
        A.aap_save(h, path)
        h2 = A.aap_load(path)
        try:
            A.aap_step(h, 6)
            A.aap_step(h2, 6)
            for u, v in zip(A.aap_get_state(h, p.n), A.aap_get_state(h2, p.n)):
                assert np.array_equal(u, v)
        finally:
            A.aap_destroy(h2)
    finally:
        A.aap_destroy(h)
    with pytest.raises(A.AapError) as e:
        A.aap_ens_create([p, p])
    assert e.value.code == A.AAP_EINVAL and "metric-free" in str(e.value)
