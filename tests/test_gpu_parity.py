"""CUDA path vs FP64 oracle, through the C ABI (needs a GB300).

Sizes span several tiles with ragged edges; every case compares element by
element with the oracle (tests/gpu_helpers.py states the tolerances).
"""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from tests import inputs
from tests.gpu_helpers import compare_one_step, oracle_model, params, wrap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _run(O, p, steps=3, state=None, max_bad_frac=0.0):
    h = A.aap_create(p)
    try:
        if state is not None:
            A.aap_set_state(h, *state, step=0)
        stats = []
        for _ in range(steps):
            stats.append(compare_one_step(O, p, h, max_bad_frac=max_bad_frac))
        return stats
    finally:
        A.aap_destroy(h)


def test_initial_state_matches_oracle(lib, oracle):
    """Philox tag-1 initial state (uniform positions, isotropic angles)."""
    p = params(n=5000, lx=41.3, ly=37.7, seed=11)
    h = A.aap_create(p)
    try:
        x, y, th = A.aap_get_state(h, p.n)
        lay = A.aap_get_layout(h)
    finally:
        A.aap_destroy(h)
    xo, yo, to = oracle.init_state(oracle_model(oracle, p))
    ux = lay.cell_x * 2.0 ** -lay.fix_bits_x
    assert np.abs(x - xo).max() <= ux and np.abs(y - yo).max() <= lay.cell_y * 2.0 ** -lay.fix_bits_y
    assert np.abs(wrap(th.astype(np.float64) - to.astype(np.float32).astype(np.float64))).max() == 0.0


@pytest.mark.parametrize("n,lx,ly,tile", [
    (2000, 33.3, 29.1, (0, 0)),      # cells slightly larger than R, ragged tiles
    (6000, 54.0, 40.0, (16, 8)),     # several tiles per axis
    (1500, 20.0, 20.0, (6, 7)),      # smallest tiles
    (300, 3.0, 4.5, (0, 0)),         # smallest box: 3 cells per axis, one tile
])
def test_vm_periodic_one_step(lib, oracle, n, lx, ly, tile):
    p = params(n=n, lx=lx, ly=ly, eta=0.4, v=0.5, seed=5, tile_w=tile[0], tile_h=tile[1])
    for s in _run(oracle, p, steps=3):
        assert s["max_dtheta_wellcond"] < 1e-5


@pytest.mark.parametrize("bx,by", [(1, 0), (0, 1), (1, 1)])
def test_vm_reflecting_one_step(lib, oracle, bx, by):
    p = params(n=3000, lx=37.5, ly=31.2, eta=0.3, v=0.7, seed=9, bx=bx, by=by)
    _run(oracle, p, steps=3)


def test_nvm_one_step(lib, oracle):
    p = params(n=4000, lx=40.0, ly=40.0, eta=0.1, v=0.5, seed=13, model=A.AAP_NVM)
    _run(oracle, p, steps=3)


@pytest.mark.parametrize("weight,order,bx,by", [(0, 1, 1, 1), (1, 1, 0, 0), (0, 2, 1, 0), (1, 3, 0, 1)])
def test_langevin_one_step(lib, oracle, weight, order, bx, by):
    """Eq. (Langevin_dynamics) with the Euler-Maruyama step, h = 1/(1+n) or 1,
    interaction order o, reflecting walls (the configuration of the Brownian
    workload: Gamma = 1, D = 0.1 so eta = sqrt(2D), dt = 0.01, v0 = 1)."""
    p = params(n=3000, lx=38.7, ly=38.7, v=1.0, eta=np.sqrt(0.2), gamma=1.0, dt=0.01,
               model=A.AAP_LANGEVIN, weight=weight, order=order, bx=bx, by=by, seed=17)
    _run(oracle, p, steps=3)


def test_chirality_and_large_steps(lib, oracle):
    p = params(n=2500, lx=35.0, ly=35.0, eta=0.25, omega=0.8, v=1.0, seed=21)
    _run(oracle, p, steps=2)


def test_dense_cluster_uses_scratch_and_spill(lib, oracle):
    """Everything in a few cells: tiles overflow shared-memory staging (global
    scratch path) and their regions (spill list); results stay exact."""
    n, L = 3000, 24.0
    x, y, th = inputs.clustered_state(n, L, L, 3, 12.2, 11.7, 2.5)
    p = params(n=n, lx=L, ly=L, eta=0.2, v=0.3, seed=23, tile_w=8, tile_h=8, capacity=1.0)
    h = A.aap_create(p)
    try:
        A.aap_set_state(h, x, y, th.astype(np.float32), step=0)
        for _ in range(2):
            compare_one_step(oracle, p, h)
        assert A.aap_observe(h).flags & A.AAP_FLAG_SPILLED
    finally:
        A.aap_destroy(h)


def test_band_state(lib, oracle):
    """A dense band (the inhomogeneous load of ordered VM states, Sec. 3.2)."""
    n, L = 8000, 50.0
    x, y, th = inputs.band_state(n, L, L, 4, 0.6, 4.0)
    p = params(n=n, lx=L, ly=L, eta=0.2, v=0.5, seed=29)
    h = A.aap_create(p)
    try:
        A.aap_set_state(h, x, y, th.astype(np.float32), step=0)
        for _ in range(2):
            compare_one_step(oracle, p, h)
    finally:
        A.aap_destroy(h)


def test_empty_and_single_particle(lib, oracle):
    p0 = params(n=0, lx=10.0, ly=10.0)
    h = A.aap_create(p0)
    A.aap_step(h, 5)
    o = A.aap_observe(h)
    assert o.phi == 0.0 and o.step == 5
    A.aap_destroy(h)
    p1 = params(n=1, lx=10.0, ly=10.0, eta=0.3, omega=0.1, seed=3)
    _run(oracle, p1, steps=4)


def test_phi_matches_oracle(lib, oracle):
    p = params(n=7000, lx=60.0, ly=60.0, seed=31)
    h = A.aap_create(p)
    try:
        tr = A.aap_phi_trace(h, 5)
        x, y, th = A.aap_get_state(h, p.n)
        assert abs(tr[-1] - oracle.polar(th.astype(np.float64))) < 1e-6
        o = A.aap_observe(h)
        assert abs(o.phi - tr[-1]) < 1e-6
        assert abs(o.q - oracle.nematic(th.astype(np.float64))) < 1e-6
    finally:
        A.aap_destroy(h)


def test_ordered_state_stays_ordered(lib):
    """eta = 0 from theta_i = theta0: p = 1 at every step (Eq. collision_VM)."""
    n, L = 20000, 100.0
    x, y, th = inputs.ordered_state(n, L, L, 5, 0.3)
    p = params(n=n, lx=L, ly=L, eta=0.0, v=0.5)
    h = A.aap_create(p)
    try:
        A.aap_set_state(h, x, y, th.astype(np.float32), step=0)
        tr = A.aap_phi_trace(h, 50)
    finally:
        A.aap_destroy(h)
    assert np.abs(tr - 1.0).max() < 1e-6


def test_deterministic_and_resume_bitwise(lib):
    """Same state -> bit-identical trajectory (region and cell order are set by
    atomics, but the neighbour sums are exact integers); k steps + get/set_state
    + rest = all steps."""
    p = params(n=20000, lx=100.0, ly=100.0, eta=0.45, seed=37)
    h1 = A.aap_create(p)
    h2 = A.aap_create(p)
    try:
        A.aap_step(h1, 20)
        A.aap_step(h2, 8)
        s = A.aap_get_state(h2, p.n)
        A.aap_set_state(h2, *s, step=8)
        A.aap_step(h2, 12)
        a = A.aap_get_state(h1, p.n)
        b = A.aap_get_state(h2, p.n)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


@pytest.mark.parametrize("threads", [512, 0])
def test_handles_of_different_staging_sizes_coexist(lib, threads):
    """A dense system (large shared-memory staging) keeps stepping after a
    sparse one (small staging) was created, and its trajectory is the one it
    has alone: the kernel's shared-memory limit is a per-process maximum.
    threads = 512: the whole-block kernel, whose staging follows the density;
    0: the pipelined kernel, whose buffers follow the tile shape (the sparse
    system's tiles are smaller here, so its launch asks for a different
    amount of shared memory)."""
    dense = params(n=40000, lx=100.0, ly=100.0, eta=0.3, seed=41, threads=threads)       # rho = 4
    sparse = params(n=2000, lx=60.0, ly=60.0, eta=0.3, seed=42, threads=threads,         # rho = 0.56
                    tile_w=0 if threads else 12, tile_h=0 if threads else 12)
    ref = A.aap_create(dense)
    try:
        A.aap_step(ref, 10)
        want = A.aap_get_state(ref, dense.n)
    finally:
        A.aap_destroy(ref)
    h1 = A.aap_create(dense)
    h2 = A.aap_create(sparse)
    try:
        l1, l2 = A.aap_get_layout(h1), A.aap_get_layout(h2)
        if threads:
            assert l1.stage_cap > l2.stage_cap
        else:
            assert l1.threads == l2.threads == 1024
        A.aap_step(h2, 5)
        A.aap_step(h1, 10)
        for u, v in zip(A.aap_get_state(h1, dense.n), want):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_long_call_grows_regions_within_the_call(lib):
    """Clustering (low noise) overflows the tile regions: one long aap_step
    call re-lays them out between its batches, and its trajectory equals the
    one of many short calls bit for bit."""
    p = params(n=1 << 18, lx=362.0, ly=362.0, eta=0.1, v=0.5, seed=61)
    h1, h2 = A.aap_create(p), A.aap_create(p)
    try:
        slots0 = A.aap_get_layout(h1).tile_slots
        A.aap_step(h1, 1536)
        A.aap_sync(h1)
        assert A.aap_get_layout(h1).tile_slots > slots0          # grown inside the one call
        assert A.aap_observe(h1).flags & A.AAP_FLAG_SPILLED
        for _ in range(12):
            A.aap_step(h2, 128)
        for u, v in zip(A.aap_get_state(h1, p.n), A.aap_get_state(h2, p.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_translation_by_whole_tiles_bitwise(lib):
    """Periodic box, shift every particle by whole tiles: the trajectory is the
    shifted trajectory bit for bit (the noise is keyed on id, not position)."""
    n, L = 12000, 128.0
    x, y, th = inputs.uniform_state(n, L, L, 8)
    p = params(n=n, lx=L, ly=L, eta=0.45, seed=41, tile_w=16, tile_h=16)
    h1 = A.aap_create(p)
    h2 = A.aap_create(p)
    try:
        A.aap_set_state(h1, x, y, th.astype(np.float32), step=0)
        sx, sy = 48.0, 80.0
        A.aap_set_state(h2, np.mod(x + sx, L), np.mod(y + sy, L), th.astype(np.float32), step=0)
        A.aap_step(h1, 10)
        A.aap_step(h2, 10)
        a = A.aap_get_state(h1, n)
        b = A.aap_get_state(h2, n)
        assert np.array_equal(a[2], b[2])
        assert np.array_equal(np.mod(a[0] + sx, L), b[0])
        assert np.array_equal(np.mod(a[1] + sy, L), b[1])
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_reflecting_mirror_extension_on_gpu(lib):
    """eta = 0: the reflecting system (x walls) equals the doubled periodic
    system of mirror copies, both run on the GPU (Sec. 2.4)."""
    n, lx, ly = 4000, 40.0, 33.0
    x, y, th = inputs.uniform_state(n, lx, ly, 12)
    pr = params(n=n, lx=lx, ly=ly, eta=0.0, v=0.5, bx=1)
    pe = params(n=2 * n, lx=2 * lx, ly=ly, eta=0.0, v=0.5)
    hr = A.aap_create(pr)
    he = A.aap_create(pe)
    try:
        A.aap_set_state(hr, x, y, th.astype(np.float32))
        xe = np.concatenate([x, 2 * lx - x])
        te = np.concatenate([th, wrap(np.pi - th)]).astype(np.float32)
        A.aap_set_state(he, xe, np.concatenate([y, y]), te)
        A.aap_step(hr, 2)
        A.aap_step(he, 2)
        a = A.aap_get_state(hr, n)
        b = A.aap_get_state(he, 2 * n)
        k = np.where(b[0][:n] <= lx, np.arange(n), np.arange(n) + n)
        assert np.abs(b[0][k] - a[0]).max() < 1e-4
        assert np.abs(wrap(b[2][k].astype(np.float64) - a[2])).max() < 1e-4
    finally:
        A.aap_destroy(hr)
        A.aap_destroy(he)


def test_full_size_sampled(lib, oracle):
    """N = 2^24, L = 2896 (rho = 2), R = 1, v0 = 0.5: steps in the launch
    configuration the benchmark times, sampled particles against the oracle.
    On the uniform initial state the mean neighbour number is
    (N-1) pi R^2 / L^2, and the fused on-the-fly sum equals the mean of the
    per-particle counts."""
    n, L = 1 << 24, 2896.0
    p = params(n=n, lx=L, ly=L, eta=0.45, v=0.5, seed=1)
    h = A.aap_create(p)
    try:
        nb0 = A.aap_step_neighbours(h, n)
        o = A.aap_observe(h)
        assert abs(o.mean_neighbours - nb0.mean()) < 1e-9
        assert abs(nb0.mean() - (n - 1) * np.pi / L**2) < 0.01
        A.aap_step(h, 1)
        idx = np.random.default_rng(0).choice(n, 3000, replace=False)
        compare_one_step(oracle, p, h, idx=idx)
    finally:
        A.aap_destroy(h)


def test_set_state_rejects_invalid_values_and_keeps_the_state(lib):
    """Positions outside the box and non-finite orientations are found on the
    device; the lowest offending index is named and the state stays as it was."""
    p = params(n=50000, lx=160.0, ly=160.0, seed=43)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        before = A.aap_get_state(h, p.n)
        step = A.aap_observe(h).step
        x, y, th = (a.copy() for a in before)
        x[31337] = p.lx + 0.5
        th[777] = np.nan
        with pytest.raises(A.AapError) as e:
            A.aap_set_state(h, x, y, th, step=0)
        assert e.value.code == A.AAP_EINVAL and "orientation 777" in str(e.value)
        th[777] = 0.25
        with pytest.raises(A.AapError) as e:
            A.aap_set_state(h, x, y, th, step=0)
        assert e.value.code == A.AAP_EINVAL and "position 31337" in str(e.value)
        assert A.aap_observe(h).step == step
        for u, v in zip(A.aap_get_state(h, p.n), before):
            assert np.array_equal(u, v)
        A.aap_step(h, 2)
        assert np.isfinite(A.aap_observe(h).phi)
    finally:
        A.aap_destroy(h)


def test_invalid_parameters_rejected(lib):
    for kw in [dict(lx=2.5), dict(n=-1), dict(v=1.5), dict(model=7), dict(eta=float("nan")),
               dict(model=A.AAP_LANGEVIN, dt=0.0), dict(threads=100), dict(tile_w=3)]:
        with pytest.raises(A.AapError) as e:
            A.aap_create(params(**kw))
        assert e.value.code == A.AAP_EINVAL
    h = A.aap_create(params(n=10, lx=10.0, ly=10.0))
    try:
        with pytest.raises(A.AapError):
            A.aap_set_state(h, np.full(10, 11.0), np.zeros(10), np.zeros(10, np.float32))
        with pytest.raises(A.AapError):
            A.aap_set_state(h, np.zeros(9), np.zeros(9), np.zeros(9, np.float32))
    finally:
        A.aap_destroy(h)


def test_long_run_time_averaged_phi_16_seeds(lib, oracle):
    """Vicsek N = 8192, L = 64, eta = 0.4, 1000 steps (the small workload):
    chaotic trajectories part ways after a few steps, so the FP32 GPU and the
    FP64 oracle are compared statistically.  Per seed 1..16, p(t) averaged over
    t in [500, 1000); the two 16-seed means agree within 3 sigma, sigma the
    standard error of their difference (sqrt(s_o^2/16 + s_g^2/16))."""
    import os

    T, seeds = 1000, range(1, 17)
    g_means, o_means = [], []
    for s in seeds:
        p = params(n=8192, lx=64.0, ly=64.0, r=1.0, v=0.5, eta=0.4, seed=s)
        h = A.aap_create(p)
        try:
            x0, y0, t0 = A.aap_get_state(h, p.n)
            phi_g = A.aap_phi_trace(h, T)
        finally:
            A.aap_destroy(h)
        m = oracle_model(oracle, p)
        phi_o = oracle.run(m, x0, y0, t0.astype(np.float64), 0, T, threads=os.cpu_count() or 1)[3]
        g_means.append(phi_g[T // 2:T].mean())
        o_means.append(phi_o[T // 2:T].mean())
    g, o = np.array(g_means), np.array(o_means)
    sigma = np.sqrt(o.var(ddof=1) / len(o) + g.var(ddof=1) / len(g))
    assert abs(o.mean() - g.mean()) < 3 * sigma, (o.mean(), g.mean(), sigma)
    assert 0.05 < g.mean() < 1.0


def test_largest_practical_system_keeps_every_particle(lib, oracle):
    """N = 2^27 (L = 8192, rho = 2; about 20 GB on the device): every record is
    kept (aap_observe counts them), p stays a valid order parameter, and sampled
    particles of a later step still match the oracle on a local copy of their
    neighbourhood."""
    p = params(n=1 << 27, lx=8192.0, ly=8192.0, eta=0.45, seed=71)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        obs = A.aap_observe(h)                   # raises if a record was lost
        assert obs.step == 3 and 0.0 <= obs.phi < 0.01
        x, y, th = A.aap_get_state(h, p.n)
        step = obs.step
        nb = A.aap_step_neighbours(h, p.n)
        x1, y1, t1 = A.aap_get_state(h, p.n)
    finally:
        A.aap_destroy(h)
    # neighbour counts of sampled particles: the oracle on the particles of a
    # 48 x 48 window centred on each (its own periodic box; the centre is far
    # from the window's edges, so only true neighbours can reach it)
    rng = np.random.default_rng(3)
    checked = 0
    for i in rng.choice(p.n, 12, replace=False):
        if not (30 < x[i] < p.lx - 30 and 30 < y[i] < p.ly - 30):
            continue
        sel = np.nonzero((np.abs(x - x[i]) < 24) & (np.abs(y - y[i]) < 24))[0]
        k = int(np.nonzero(sel == i)[0][0])
        m = oracle_model(oracle, params(n=sel.size, lx=48.0, ly=48.0, eta=p.eta, seed=p.seed))
        xs, ys = x[sel] - (x[i] - 24.0), y[sel] - (y[i] - 24.0)
        _, _, _, nbo, _, amb = oracle.step(m, xs, ys, th[sel].astype(np.float64), step, idx=np.array([k]))
        if amb[0]:
            continue
        assert nb[i] == nbo[0]
        checked += 1
    assert checked >= 8
