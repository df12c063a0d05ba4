"""Batched ensembles, on-the-fly measurements, coarse-graining and graph replay
(CUDA path through the C ABI; needs a GB300)."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from paper_2211_15630_gb300 import workloads as W
from oracle import coarse as CG
from tests.gpu_helpers import compare_one_step, oracle_model, params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _standalone_like(e, r, p):
    lay = A.aap_ens_get_layout(e, r)
    q = A.aap_params_default()
    for f, _ in A.aap_params._fields_:
        setattr(q, f, getattr(p, f))
    q.tile_w, q.tile_h = lay.tile_w, lay.tile_h
    return q


def test_graph_replay_equals_single_steps(lib):
    """aap_step(h, 100) replays a captured CUDA graph of 32 steps; the
    trajectory is bit-identical to 100 single-step calls."""
    p = params(n=30000, lx=120.0, ly=120.0, eta=0.45, seed=3)
    h1, h2 = A.aap_create(p), A.aap_create(p)
    try:
        A.aap_step(h1, 100)
        for _ in range(100):
            A.aap_step(h2, 1)
        for u, v in zip(A.aap_get_state(h1, p.n), A.aap_get_state(h2, p.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_ensemble_grows_replica_regions_within_a_call(lib):
    """Low-noise replicas cluster and overflow their regions during one long
    aap_ens_step call: the ensemble re-lays them out between its batches
    (the replica's slots grow) and still follows the standalone trajectories
    bit for bit."""
    ps = []
    for r in range(4):
        q = params(n=1 << 16, lx=181.0, ly=181.0, eta=0.1 + 0.05 * r, v=0.5, seed=300 + r)
        q.tile_w, q.tile_h = 32, 16
        ps.append(q)
    e = A.aap_ens_create(ps)
    try:
        slots0 = [A.aap_ens_get_layout(e, r).tile_slots for r in range(4)]
        A.aap_ens_step(e, 1024)          # re-layouts happen on the host inside this call
        grown = [A.aap_ens_get_layout(e, r).tile_slots > slots0[r] for r in range(4)]
        assert any(grown)
        for r in range(4):
            q = _standalone_like(e, r, ps[r])
            h = A.aap_create(q)
            try:
                A.aap_step(h, 1024)
                for u, v in zip(A.aap_get_state(h, q.n), A.aap_ens_get_state(e, r, q.n)):
                    assert np.array_equal(u, v)
            finally:
                A.aap_destroy(h)
    finally:
        A.aap_ens_destroy(e)


def test_ensemble_replicas_bitwise_equal_standalone(lib):
    """Every replica of the batched launch follows the standalone trajectory
    bit for bit (same parameters, same tile shape)."""
    ps = W.ensemble_replicas(count=12, seed=7, nmin_log2=9, nmax_log2=14)
    e = A.aap_ens_create(ps)
    try:
        A.aap_ens_step(e, 40)
        for r in (0, 3, 7, 11):
            q = _standalone_like(e, r, ps[r])
            h = A.aap_create(q)
            try:
                A.aap_step(h, 40)
                a = A.aap_get_state(h, q.n)
                b = A.aap_ens_get_state(e, r, q.n)
                for u, v in zip(a, b):
                    assert np.array_equal(u, v), f"replica {r} differs"
            finally:
                A.aap_destroy(h)
    finally:
        A.aap_ens_destroy(e)


def test_ensemble_replica_matches_oracle(lib, oracle):
    """One replica's next step, taken inside the ensemble, against the oracle."""
    ps = W.ensemble_replicas(count=6, seed=11, nmin_log2=10, nmax_log2=13)
    e = A.aap_ens_create(ps)
    try:
        A.aap_ens_step(e, 5)
        r = 2
        p = ps[r]
        x0, y0, t0 = A.aap_ens_get_state(e, r, p.n)
        A.aap_ens_step(e, 1)
        x1, y1, t1 = A.aap_ens_get_state(e, r, p.n)
        m = oracle.Model(n=p.n, lx=p.lx, ly=p.ly, r=p.r, v=p.v, eta=p.eta, seed=p.seed)
        xo, yo, to, nbo, smag, amb = oracle.step(m, x0, y0, t0.astype(np.float64), 5)
        ok = (amb == 0) & (smag > 0.05)
        dth = np.abs(np.mod(t1[ok] - to[ok] + np.pi, 2 * np.pi) - np.pi)
        assert dth.max() < 1e-5
    finally:
        A.aap_ens_destroy(e)


def test_ensemble_measure_and_autotune(lib):
    """Autotune resets to the initial state with the fastest policy; the time
    averaged p of a replica equals its standalone measurement bit for bit."""
    ps = W.ensemble_replicas(count=10, seed=5, nmin_log2=10, nmax_log2=14)
    e = A.aap_ens_create(ps)
    try:
        pol, ms = A.aap_ens_autotune(e, 5)
        assert 0 <= pol < 8 and ms[pol] > 0 and ms[pol] == ms[ms > 0].min()
        A.aap_ens_step(e, 20)
        A.aap_ens_measure(e, 30)
        phi = A.aap_ens_phi_mean(e)
        assert ((phi > 0) & (phi <= 1)).all()
        r = 4
        q = _standalone_like(e, r, ps[r])
        q.threads = A.ENS_POLICIES[pol][0]
        h = A.aap_create(q)
        try:
            A.aap_step(h, 20)
            A.aap_measure(h, 30)
            res = A.aap_get_results(h)
            assert res.samples == 30
            assert res.p[0] == phi[r]
            er = A.aap_ens_results(e, r)
            assert er.samples == 30 and er.binder == res.binder
        finally:
            A.aap_destroy(h)
    finally:
        A.aap_ens_destroy(e)


def test_measurement_window_matches_trace(lib):
    """aap_measure(n) samples the states t0 .. t0+n-1 (Sec. 3.4): its <p> and
    <p^2> equal the moments of the p(t) trace of an identical system."""
    p = params(n=20000, lx=100.0, ly=100.0, eta=0.3, seed=9)
    h1, h2 = A.aap_create(p), A.aap_create(p)
    try:
        A.aap_step(h1, 10)
        A.aap_step(h2, 10)
        A.aap_measure(h1, 25)
        res = A.aap_get_results(h1)
        tr = A.aap_phi_trace(h2, 25)[:25]
        assert res.samples == 25
        assert abs(res.p[0] - tr.mean()) < 1e-12
        assert abs(res.p[1] - (tr**2).mean()) < 1e-12
        assert abs(res.binder - (1 - (tr**4).mean() / (3 * (tr**2).mean() ** 2))) < 1e-9
        assert 0 < res.nbar[0] < 50 and 0 <= res.q[0] <= 1
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_coarse_grain_conserves(lib, oracle):
    """Binned density integrates to N exactly, binned polarisation to
    sum e^{i theta}, so p follows from the fields (128 x 128 bins, 4 x 4 units)."""
    torch = pytest.importorskip("torch")
    p = W.surrogate_training(eta=0.4, seed=10000)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 10)
        out = torch.zeros(3 * 128 * 128, dtype=torch.float32, device="cuda")
        A.aap_coarse_grain(h, 128, 128, out.data_ptr())
        A.aap_sync(h)
        f = out.cpu().numpy().reshape(3, 128, 128).astype(np.float64)
        area = (p.lx / 128) * (p.ly / 128)
        assert abs(f[0].sum() * area - p.n) < 1e-3 * 1e-3 * p.n
        assert np.allclose(f[0] * area, np.round(f[0] * area), atol=1e-3)
        x, y, th = A.aap_get_state(h, p.n)
        cs = np.cos(th.astype(np.float64)).sum()
        sn = np.sin(th.astype(np.float64)).sum()
        assert abs(f[1].sum() * area - cs) < 1e-3 * np.sqrt(p.n)
        assert abs(f[2].sum() * area - sn) < 1e-3 * np.sqrt(p.n)
        assert np.array_equal(np.round(f[0] * area), CG.counts(x, y, p.lx, p.ly, 128, 128))
        ref = CG.coarse_grain(x, y, th, p.lx, p.ly, 128, 128)
        assert np.all(np.abs(f[1:] - ref[1:]) * area < 1e-6 * (np.round(ref[0] * area) + 1.0))
        phi_f = np.hypot(f[1].sum(), f[2].sum()) * area / p.n
        assert abs(phi_f - oracle.polar(th.astype(np.float64))) < 1e-6
    finally:
        A.aap_destroy(h)


@pytest.mark.parametrize("lx,ly,nbx,nby,bx", [(300.0, 210.0, 77, 53, 0), (150.0, 97.0, 211, 13, 1)])
def test_coarse_grain_exact_bins_odd_geometry(lib, lx, ly, nbx, nby, bx):
    """Bin widths that are not powers of two (and, second case, bins finer
    than the cells in x, reflecting walls): every particle's bin is
    floor(x nbx / L) of its FP64 position, so the counts equal numpy's exactly;
    the polarisation sums agree with FP64 cos / sin to FP32 rounding."""
    torch = pytest.importorskip("torch")
    p = params(n=int(2 * lx * ly), lx=lx, ly=ly, eta=0.4, seed=17, bx=bx, by=bx)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 6)
        out = torch.zeros(3 * nbx * nby, dtype=torch.float32, device="cuda")
        A.aap_coarse_grain(h, nbx, nby, out.data_ptr())
        A.aap_sync(h)
        f = out.cpu().numpy().reshape(3, nby, nbx).astype(np.float64)
        area = (lx / nbx) * (ly / nby)
        x, y, th = A.aap_get_state(h, p.n)
        ref = CG.coarse_grain(x, y, th, lx, ly, nbx, nby)
        counts = CG.counts(x, y, lx, ly, nbx, nby)
        assert np.array_equal(np.round(f[0] * area), counts)
        tol = 1e-6 * (counts + 1.0)
        assert np.all(np.abs(f[1:] - ref[1:]) * area < tol)
    finally:
        A.aap_destroy(h)


def test_coarse_grain_with_spilled_records(lib):
    """A clustered state with an explicit capacity keeps particles in the spill
    list: the fields still count every particle in its FP64 bin."""
    torch = pytest.importorskip("torch")
    from tests import inputs
    n, L, nb = 3000, 24.0, 6
    x, y, th = inputs.clustered_state(n, L, L, 3, 12.2, 11.7, 2.5)
    p = params(n=n, lx=L, ly=L, eta=0.2, v=0.3, seed=23, tile_w=8, tile_h=8, capacity=1.0)
    h = A.aap_create(p)
    try:
        A.aap_set_state(h, x, y, th.astype(np.float32), step=0)
        A.aap_step(h, 1)
        assert A.aap_observe(h).flags & A.AAP_FLAG_SPILLED
        out = torch.zeros(3 * nb * nb, dtype=torch.float32, device="cuda")
        A.aap_coarse_grain(h, nb, nb, out.data_ptr())
        A.aap_sync(h)
        f = out.cpu().numpy().reshape(3, nb, nb).astype(np.float64)
        xs, ys, ts = A.aap_get_state(h, n)
        counts = CG.counts(xs, ys, L, L, nb, nb)
        area = (L / nb) ** 2
        assert np.array_equal(np.round(f[0] * area), counts)
        ref = CG.coarse_grain(xs, ys, ts, L, L, nb, nb)
        assert np.all(np.abs(f[1:] - ref[1:]) * area < 1e-6 * (counts + 1.0))
    finally:
        A.aap_destroy(h)


def test_brownian_workload_one_step(lib, oracle):
    """The Brownian workload (N = 2^20, 724 x 724, reflecting walls, dt = 0.01):
    sampled one-step parity in the launch configuration of the benchmark."""
    p = W.brownian_walls(seed=3)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 3)
        idx = np.random.default_rng(2).choice(p.n, 3000, replace=False)
        compare_one_step(oracle, p, h, idx=idx)
    finally:
        A.aap_destroy(h)


def _theta_bins(th, bins):
    """Bin of theta in [-pi, pi) with the kernel's FP32 operations (an integer
    decided by floating point is decided in the same precision on both sides)."""
    t = th.astype(np.float32)
    k = np.float32(bins) * (np.float32(1.0) / np.float32(6.28318530717959))
    b = np.floor((t + np.float32(3.14159265358979)) * k).astype(np.int64)
    return np.clip(b, 0, bins - 1)


@pytest.mark.parametrize("bins_nbr", [64, 5])
def test_histograms_match_sampled_states(lib, oracle, bins_nbr):
    """Histograms of theta and of |Omega_i| over the measured states t0 ..
    t0+n-1 (Sec. 3.4) equal those of the same states read back one by one:
    theta bins exactly, neighbour numbers against the oracle's counts up to
    pairs within 1e-5 of the radius; the last neighbour bin collects the rest."""
    p = params(n=12000, lx=80.0, ly=80.0, eta=0.35, seed=17)
    p.binnum_theta, p.binnum_neighbors = 36, bins_nbr
    m = oracle_model(oracle, p)
    h1, h2 = A.aap_create(p), A.aap_create(p)
    nmeas = 6
    try:
        A.aap_step(h1, 9)
        A.aap_step(h2, 9)
        A.aap_measure(h1, nmeas)
        th_h, nb_h = A.aap_get_histograms(h1, 36, bins_nbr)
        res = A.aap_get_results(h1)
        ct = np.zeros(36, np.int64)
        cn = np.zeros(bins_nbr, np.int64)
        amb_total = 0
        for _ in range(nmeas):
            x, y, th = A.aap_get_state(h2, p.n)
            step = A.aap_observe(h2).step
            ct += np.bincount(_theta_bins(th, 36), minlength=36)
            _, _, _, nb, _, amb = oracle.step(m, x, y, th.astype(np.float64), step)
            amb_total += int((amb != 0).sum())
            cn += np.bincount(np.minimum(nb, bins_nbr - 1), minlength=bins_nbr)
            A.aap_step(h2, 1)
        total = p.n * nmeas
        assert np.array_equal(np.rint(th_h * total).astype(np.int64), ct)
        assert abs(th_h.sum() - 1) < 1e-12 and abs(nb_h.sum() - 1) < 1e-12
        got = np.rint(nb_h * total).astype(np.int64)
        assert np.abs(got - cn).sum() <= 2 * amb_total
        if bins_nbr == 64 and cn[-1] == 0:
            # unclipped: the histogram's mean is the measured mean neighbour number
            assert abs((np.arange(bins_nbr) * nb_h).sum() - res.nbar[0]) < 1e-9
        A.aap_clear_results(h1)
        th0, nb0 = A.aap_get_histograms(h1, 36, bins_nbr)
        assert not th0.any() and not nb0.any()
        with pytest.raises(A.AapError):
            A.aap_get_histograms(h1, 35, bins_nbr)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)


def test_save_load_continues_bitwise(lib, tmp_path):
    """A system saved after a measurement and loaded into a new handle carries
    on bit for bit, with the saved moments and histograms."""
    p = params(n=25000, lx=110.0, ly=110.0, eta=0.3, seed=23, model=A.AAP_LANGEVIN, dt=0.1, v=0.5)
    p.binnum_theta, p.binnum_neighbors = 24, 40
    h = A.aap_create(p)
    path = str(tmp_path / "sys.aap")
    try:
        A.aap_step(h, 7)
        A.aap_measure(h, 5)
        A.aap_save(h, path)
        h2 = A.aap_load(path)
        try:
            r1, r2 = A.aap_get_results(h), A.aap_get_results(h2)
            assert r1.samples == r2.samples == 5 and list(r1.p) == list(r2.p) and list(r1.nbar) == list(r2.nbar)
            for u, v in zip(A.aap_get_histograms(h, 24, 40), A.aap_get_histograms(h2, 24, 40)):
                assert np.array_equal(u, v)
            assert A.aap_observe(h2).step == A.aap_observe(h).step == 12
            A.aap_step(h, 9)
            A.aap_step(h2, 9)
            for u, v in zip(A.aap_get_state(h, p.n), A.aap_get_state(h2, p.n)):
                assert np.array_equal(u, v)
            assert A.aap_observe(h).phi == A.aap_observe(h2).phi
        finally:
            A.aap_destroy(h2)
    finally:
        A.aap_destroy(h)
