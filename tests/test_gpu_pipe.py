"""The pipelined step kernel (threads = 1024: copy, sort and update warps with
mbarrier hand-offs) against the whole-block step kernel (threads = 512) and
the FP64 oracle, through the C ABI (needs a GB300).

Both kernels compute the same neighbour sums in exact integers and the same
per-particle FP32 arithmetic, so their trajectories must agree bit for bit,
whatever order the tiles and particles are processed in; the one-step
comparisons with the oracle use the tolerances of tests/gpu_helpers.py."""
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


def _pair(p, state=None):
    q = A.aap_params_default()
    for f, _ in A.aap_params._fields_:
        setattr(q, f, getattr(p, f))
    p.threads, q.threads = 1024, 512
    h1, h2 = A.aap_create(p), A.aap_create(q)
    if state is not None:
        for h in (h1, h2):
            A.aap_set_state(h, *state, step=0)
    return h1, h2


def _same(h1, h2, n):
    a = A.aap_get_state(h1, n)
    b = A.aap_get_state(h2, n)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    o1, o2 = A.aap_observe(h1), A.aap_observe(h2)
    assert o1.step == o2.step and o1.phi == o2.phi and o1.q == o2.q
    assert o1.mean_neighbours == o2.mean_neighbours


def test_default_layout_is_pipelined(lib):
    p = params(n=20000, lx=100.0, ly=100.0, seed=3)
    h = A.aap_create(p)
    try:
        lay = A.aap_get_layout(h)
        assert lay.threads == 1024 and lay.stage_cap >= 1024
    finally:
        A.aap_destroy(h)
    with pytest.raises(A.AapError):
        A.aap_create(params(n=100, lx=20.0, ly=20.0, threads=1024, kn=4))


@pytest.mark.parametrize("case", ["vm", "vm_ragged_tiles", "nvm", "langevin_walls", "langevin_o2", "smallest_box"])
def test_pipelined_equals_block_kernel(lib, case):
    kw = {
        "vm": dict(n=60000, lx=173.0, ly=171.0, eta=0.45, v=0.5),
        "vm_ragged_tiles": dict(n=9000, lx=70.3, ly=61.7, eta=0.3, v=0.5, tile_w=13, tile_h=9),
        "nvm": dict(n=20000, lx=100.0, ly=100.0, eta=0.2, v=0.5, model=A.AAP_NVM),
        "langevin_walls": dict(n=20000, lx=100.0, ly=100.0, v=1.0, eta=np.sqrt(0.2), gamma=1.0, dt=0.01,
                               model=A.AAP_LANGEVIN, bx=1, by=1),
        "langevin_o2": dict(n=12000, lx=80.0, ly=75.0, v=1.0, eta=0.4, gamma=1.5, dt=0.05,
                            model=A.AAP_LANGEVIN, order=2, weight=A.AAP_H_ONE, bx=1),
        "smallest_box": dict(n=300, lx=3.0, ly=4.5, eta=0.4, v=0.5),
    }[case]
    p = params(seed=41, **kw)
    h1, h2 = _pair(p)
    try:
        for k in (1, 4, 45):
            A.aap_step(h1, k)
            A.aap_step(h2, k)
            _same(h1, h2, p.n)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


@pytest.mark.parametrize("n,w", [(3200, 7.0), (5000, 4.0), (12000, 3.0)])
def test_pipelined_dense_tiles(lib, oracle, n, w):
    """A cluster denser than a tile's shared buffers hold: up to twice their
    capacity a tile goes through the pipeline as one wide tile over both
    buffers (first case), beyond that to the whole-block routine at the end of
    the pipelined kernel (its shared staging area, or global scratch for the
    last case); the result equals the block kernel's bit for bit and the
    oracle's within tolerance."""
    L = 64.0
    x, y, th = inputs.clustered_state(n, L, L, 7, 30.5, 33.2, w)
    p = params(n=n, lx=L, ly=L, eta=0.2, v=0.3, seed=43)
    h1, h2 = _pair(p, (x, y, th.astype(np.float32)))
    try:
        lay = A.aap_get_layout(h1)
        assert lay.threads == 1024 and n > lay.stage_cap
        compare_one_step(oracle, p, h1)
        A.aap_step_neighbours(h2, n)
        _same(h1, h2, n)
        for k in (1, 10):
            A.aap_step(h1, k)
            A.aap_step(h2, k)
            _same(h1, h2, n)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_pipelined_spilled_records(lib, oracle):
    """Small tiles at capacity factor 1: records spill out of their regions
    and the pipelined kernel's copy warp stages them from the spill list (or
    leaves the tile to the whole-block routine when too many match)."""
    n, L = 3000, 24.0
    x, y, th = inputs.clustered_state(n, L, L, 3, 12.2, 11.7, 2.5)
    p = params(n=n, lx=L, ly=L, eta=0.2, v=0.3, seed=23, tile_w=8, tile_h=8, capacity=1.0)
    h1, h2 = _pair(p, (x, y, th.astype(np.float32)))
    try:
        assert A.aap_get_layout(h1).threads == 1024
        compare_one_step(oracle, p, h1)
        A.aap_step_neighbours(h2, n)
        _same(h1, h2, n)
        assert A.aap_observe(h1).flags & A.AAP_FLAG_SPILLED
        for k in (1, 6):
            A.aap_step(h1, k)
            A.aap_step(h2, k)
            _same(h1, h2, n)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_pipelined_measurements_equal(lib):
    """On-the-fly moments and histograms (Sec. 3.4) are summed per block in
    the pipelined kernel and per tile in the block kernel: same integers."""
    p = params(n=30000, lx=122.0, ly=122.0, eta=0.35, v=0.5, seed=47)
    h1, h2 = _pair(p)
    try:
        for h in (h1, h2):
            A.aap_measure(h, 60)
        r1, r2 = A.aap_get_results(h1), A.aap_get_results(h2)
        for f in ("p", "q", "nbar"):
            assert np.array_equal(np.asarray(getattr(r1, f)), np.asarray(getattr(r2, f)))
        for u, v in zip(A.aap_get_histograms(h1, 100, 100), A.aap_get_histograms(h2, 100, 100)):
            assert np.array_equal(u, v)
        _same(h1, h2, p.n)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_pipelined_full_size_sample(lib, oracle):
    """The N = 2^24, L = 2896 workload in the launch configuration the bench
    times: a few steps, then one step of 3000 sampled particles against the
    oracle (brute force over the sampled particles' neighbourhoods)."""
    from paper_2211_15630_gb300 import workloads as W

    p = W.vicsek_large(seed=1)
    h = A.aap_create(p)
    try:
        assert A.aap_get_layout(h).threads == 1024
        A.aap_step(h, 5)
        idx = np.random.default_rng(5).choice(p.n, 3000, replace=False)
        compare_one_step(oracle, p, h, idx=idx)
    finally:
        A.aap_destroy(h)


def test_pipelined_ensemble_equals_block_kernel(lib):
    """An ensemble of replicas of different sizes, densities and noise runs
    through the pipelined kernel (one launch over all replicas' tiles, each
    output buffer carrying its tile's system) and through the whole-block
    kernel: every replica's state, measured moments and time-averaged p agree
    bit for bit."""
    from paper_2211_15630_gb300 import workloads as W

    ps = W.ensemble_replicas(count=12, seed=9, nmin_log2=8.0, nmax_log2=15.0)
    qs = W.ensemble_replicas(count=12, seed=9, nmin_log2=8.0, nmax_log2=15.0, threads=512)
    e1, e2 = A.aap_ens_create(ps), A.aap_ens_create(qs)
    try:
        assert A.aap_ens_get_layout(e1, 0).threads == 1024 and A.aap_ens_get_layout(e2, 0).threads == 512
        for e in (e1, e2):
            A.aap_ens_step(e, 7)
            A.aap_ens_measure(e, 40)
        assert np.array_equal(A.aap_ens_phi_mean(e1), A.aap_ens_phi_mean(e2))
        for r, p in enumerate(ps):
            a, b = A.aap_ens_results(e1, r), A.aap_ens_results(e2, r)
            for f in ("p", "q", "nbar"):
                assert np.array_equal(np.asarray(getattr(a, f)), np.asarray(getattr(b, f))), (r, f)
            for u, v in zip(A.aap_ens_get_state(e1, r, p.n), A.aap_ens_get_state(e2, r, p.n)):
                assert np.array_equal(u, v), r
    finally:
        A.aap_ens_destroy(e1)
        A.aap_ens_destroy(e2)
