"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test names what fixes the expected value: a library routine (cuRAND's
host Philox generator, scipy's k-d tree), a closed form of the model
equations, or an invariant of the dynamics.
"""
import ctypes
import math
import os

import numpy as np
import pytest

from tests import inputs

scipy = pytest.importorskip("scipy")
from scipy import stats  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402


# ---------------------------------------------------------------- Philox ----

def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_host_philox(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 12345, 0xDEADBEEFCAFEF00D, 2**64 - 1])
def test_philox_matches_curand_host_generator(oracle, seed):
    """cuRAND's CPU Philox4x32-10 generator lays its output out as
    out[4 (65536 k + t) + w] = Philox(ctr=(k, kh, t, 0), key=(seed_lo, seed_hi))[w];
    an offset of 4 (65536 (2^32 kh + k) + t) < 2^64 starts at that block.  This pins
    the round function, both multipliers, the key schedule and counter words 0-2."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = _curand_host_philox(lib, seed, 0, 4 * 65536 * 2)
    g = np.random.default_rng(seed % 1000)
    for blk in g.integers(0, 2 * 65536, 200):
        k, t = divmod(int(blk), 65536)
        got = oracle.philox4x32_10([k, 0, t, 0], key)
        assert (got == out[4 * blk: 4 * blk + 4]).all()
    for kh, k, t in [(5, 3, 7), (1, 0, 0), (0x3FFF, 0xFFFFFFF0, 65535), (77, 123456789, 4242)]:
        off = 4 * (65536 * ((kh << 32) + k) + t)
        ref = _curand_host_philox(lib, seed, off, 4)
        assert (oracle.philox4x32_10([k, kh, t, 0], key) == ref).all()


def test_u01_exact_and_open(oracle):
    """u = ((w >> 9) + 1/2) 2^-23 lies in (0,1); u and 2u - 1 are exact in FP32."""
    for w in [0, 1, 255, 256, 0x7FFFFFFF, 0xFFFFFF00, 0xFFFFFFFF, 123456789]:
        u = oracle.u01(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert float(np.float32(2 * u - 1)) == 2 * u - 1
        k = u * 2**23 - 0.5
        assert k == math.floor(k) and k == (w >> 9)


def test_uniform_draws_chi2(oracle):
    """Uniforms of consecutive particle ids pass a 64-bin chi-square test."""
    m = oracle.Model(n=1, lx=10, ly=10, seed=99)
    u = np.array([oracle.u01(oracle.draw(m, i, 17, 0)[0]) for i in range(20000)])
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-4


def test_init_state_uniform_isotropic(oracle):
    """Initial state: positions U(0,L), angles U(-pi,pi) (Fig. runtime caption)."""
    m = oracle.Model(n=20000, lx=40.0, ly=25.0, seed=3)
    x, y, th = oracle.init_state(m)
    assert (x > 0).all() and (x < m.lx).all() and (y > 0).all() and (y < m.ly).all()
    assert (th > -np.pi).all() and (th < np.pi).all()
    assert stats.kstest(x / m.lx, "uniform").pvalue > 1e-4
    assert stats.kstest(y / m.ly, "uniform").pvalue > 1e-4
    assert stats.kstest((th + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4


# ----------------------------------------------------------- geometry -------

@pytest.mark.parametrize("L,R,nc", [(64.0, 1.0, 64), (10.5, 1.0, 10), (3.0, 1.0, 3), (7.9, 2.5, 3)])
def test_cell_geometry(oracle, L, R, nc):
    """Cells tile the box with side L/floor(L/R) >= R (Sec. 3.2)."""
    ncx, ncy, csx, csy = oracle.geometry(oracle.Model(n=1, lx=L, ly=L, r=R))
    assert ncx == nc and ncy == nc
    assert csx >= R and abs(csx * ncx - L) < 1e-12


def test_cell_geometry_rejects_small_box(oracle):
    with pytest.raises(ValueError):
        oracle.geometry(oracle.Model(n=1, lx=2.9, ly=10, r=1.0))


# ----------------------------------------------------------- neighbours -----

def _mirror_extension(x, y, th, lx, ly, bx, by):
    """Copies of a reflecting system that make it periodic on the doubled box."""
    xs, ys, ts = [x], [y], [th]
    if bx:
        xs.append(2 * lx - x); ys.append(y); ts.append(np.pi - th)
    if by:
        xs.append(x); ys.append(2 * ly - y); ts.append(-th)
    if bx and by:
        xs.append(2 * lx - x); ys.append(2 * ly - y); ts.append(th + np.pi)
    ts = [np.mod(t + np.pi, 2 * np.pi) - np.pi for t in ts]
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ts)


def _kdtree_counts(x, y, box, R, n_real):
    tree = cKDTree(np.c_[x, y], boxsize=box)
    lists = tree.query_ball_point(np.c_[x[:n_real], y[:n_real]], R)
    return np.array([len(lst) - 1 for lst in lists])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_neighbours_periodic_match_kdtree(oracle, seed):
    """Eq. (metric_neighborhood) with periodic images = scipy periodic k-d tree."""
    lx, ly, n = 12.0, 9.5, 400
    x, y, _ = inputs.uniform_state(n, lx, ly, seed)
    m = oracle.Model(n=n, lx=lx, ly=ly)
    ref = _kdtree_counts(x, y, [lx, ly], 1.0, n)
    assert (oracle.counts_brute(m, x, y) == ref).all()
    assert (oracle.counts_cell(m, x, y) == ref).all()


@pytest.mark.parametrize("bx,by", [(1, 0), (0, 1), (1, 1)])
def test_neighbours_reflecting_match_mirror_extension(oracle, bx, by):
    """Reflecting walls with image particles (Sec. 2.4) = the periodic system on
    the doubled box built from mirror copies, counted by scipy's k-d tree.  This
    pins the reading that a particle's own mirror image is a neighbour."""
    lx, ly, n = 8.0, 7.0, 300
    x, y, th = inputs.uniform_state(n, lx, ly, 11 + bx + 2 * by)
    # put some particles right at the walls so own images matter
    x[:20] = np.linspace(0.01, 0.45, 20); y[20:40] = ly - np.linspace(0.01, 0.45, 20)
    m = oracle.Model(n=n, lx=lx, ly=ly, bx=bx, by=by)
    xe, ye, _ = _mirror_extension(x, y, th, lx, ly, bx, by)
    box = [lx * (2 if bx else 1), ly * (2 if by else 1)]
    ref = _kdtree_counts(xe, ye, box, 1.0, n)
    assert (oracle.counts_brute(m, x, y) == ref).all()
    assert (oracle.counts_cell(m, x, y) == ref).all()
    m0 = oracle.Model(n=n, lx=lx, ly=ly, bx=bx, by=by, self_image=0)
    assert (oracle.counts_brute(m0, x, y) != ref).any()


def test_mean_neighbour_number_uniform(oracle):
    """Uniform states: E|Omega_i| = (N-1) pi R^2 / (Lx Ly)."""
    lx = ly = 40.0
    n = 3200
    means = []
    for s in range(8):
        x, y, _ = inputs.uniform_state(n, lx, ly, 100 + s)
        means.append(oracle.counts_cell(oracle.Model(n=n, lx=lx, ly=ly), x, y).mean())
    expect = (n - 1) * np.pi / (lx * ly)
    se = np.std(means, ddof=1) / np.sqrt(len(means))
    assert abs(np.mean(means) - expect) < 4 * max(se, 1e-3)


# -------------------------------------------------------------- VM rule -----

def _wrap(a):
    return np.mod(a + np.pi, 2 * np.pi) - np.pi


def test_vm_single_particle_closed_form(oracle):
    """N = 1: theta' = theta + omega + eta pi (2u - 1), x' = x + v cos theta'
    (Eq. collision_VM with an empty neighbourhood, Eq. streaming)."""
    m = oracle.Model(n=1, lx=6.0, ly=6.0, v=0.7, eta=0.3, omega=0.2, seed=5)
    x, y, th = np.array([3.0]), np.array([2.0]), np.array([1.1])
    for step in [0, 1, 2**33 + 7]:
        u = oracle.u01(oracle.draw(m, 0, step, 0)[0])
        xo, yo, to, nb, _, _ = oracle.step(m, x, y, th, step)
        t = 1.1 + 0.2 + 0.3 * np.pi * (2 * u - 1)
        assert nb[0] == 0
        assert abs(to[0] - _wrap(t)) < 1e-14
        assert abs(xo[0] - (3.0 + 0.7 * np.cos(t))) < 1e-14
        assert abs(yo[0] - (2.0 + 0.7 * np.sin(t))) < 1e-14


@pytest.mark.parametrize("a,b", [(0.1, 0.9), (-2.0, 2.5), (3.0, -3.0), (1.0, 1.0)])
def test_vm_two_particles_take_circular_mean(oracle, a, b):
    """Two particles within R at eta = 0: both move along the circular mean."""
    m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.5, eta=0.0)
    x, y, th = np.array([5.0, 5.4]), np.array([5.0, 5.3]), np.array([a, b])
    _, _, to, nb, _, _ = oracle.step(m, x, y, th, 0)
    mean = math.atan2(math.sin(a) + math.sin(b), math.cos(a) + math.cos(b))
    if abs(b - a) < np.pi:
        assert abs(_wrap(mean - (a + b) / 2)) < 1e-12
    assert (nb == 1).all()
    assert np.allclose(np.abs(_wrap(to - mean)), 0.0, atol=1e-12)


def test_vm_ordered_state_stays_ordered_and_translates(oracle):
    """eta = 0 from theta_i = theta0: p = 1 at all times and every particle
    moves rigidly, x(t) = x0 + t v cos theta0 (mod L)."""
    n, L, theta0, v, T = 400, 20.0, 0.3, 0.5, 25
    x, y, th = inputs.ordered_state(n, L, L, 7, theta0)
    m = oracle.Model(n=n, lx=L, ly=L, v=v, eta=0.0)
    xo, yo, to, phi = oracle.run(m, x, y, th, 0, T)
    assert np.allclose(phi, 1.0, atol=1e-12)
    assert np.allclose(to, theta0, atol=1e-12)
    dx = np.mod(xo - (x + T * v * np.cos(theta0)) + L / 2, L) - L / 2
    dy = np.mod(yo - (y + T * v * np.sin(theta0)) + L / 2, L) - L / 2
    assert np.abs(dx).max() < 1e-10 and np.abs(dy).max() < 1e-10


def test_vm_chirality_rotates_ordered_state(oracle):
    """eta = 0, omega != 0: an ordered state rotates rigidly, theta(t) = theta0 + t omega."""
    n, L, T, om = 200, 15.0, 12, 0.25
    x, y, th = inputs.ordered_state(n, L, L, 8, 0.3)
    _, _, to, phi = oracle.run(oracle.Model(n=n, lx=L, ly=L, eta=0.0, omega=om), x, y, th, 0, T)
    assert np.allclose(phi, 1.0, atol=1e-12)
    assert np.abs(_wrap(to - (0.3 + T * om))).max() < 1e-11


def test_nvm_anti_aligned_pair(oracle):
    """NVM (Eq. collision_NVM): a neighbour more than pi/2 away enters as its
    reversed direction, so an anti-aligned pair keeps its axis at eta = 0."""
    m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, eta=0.0, model=oracle.NVM)
    a, b = 0.2, 0.2 + np.pi - 0.4
    _, _, to, _, _, _ = oracle.step(m, np.array([5.0, 5.5]), np.array([5.0, 5.0]), np.array([a, b]), 0)
    ea = math.atan2(math.sin(a) + math.sin(b + np.pi), math.cos(a) + math.cos(b + np.pi))
    eb = math.atan2(math.sin(b) + math.sin(a + np.pi), math.cos(b) + math.cos(a + np.pi))
    assert abs(_wrap(to[0] - ea)) < 1e-12 and abs(_wrap(to[1] - eb)) < 1e-12
    # an aligned-enough pair behaves like the VM
    vm = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, eta=0.0)
    th = np.array([0.2, 1.0])
    a1 = oracle.step(m, np.array([5.0, 5.5]), np.array([5.0, 5.0]), th, 0)[2]
    a2 = oracle.step(vm, np.array([5.0, 5.5]), np.array([5.0, 5.0]), th, 0)[2]
    assert np.allclose(a1, a2, atol=1e-14)


# -------------------------------------------------------- Langevin rule -----

def test_langevin_free_rotational_diffusion(oracle):
    """Gamma = 0, v = 0: theta performs Brownian motion with drift omega, so
    each EM increment is N(omega dt, eta^2 dt) and <cos(theta(t)-theta(0)-omega t)>
    = exp(-eta^2 t / 2) (Eq. Langevin_dynamics with additive noise)."""
    n, L, eta, dt, om, T = 4000, 200.0, 0.8, 0.05, 0.3, 40
    x, y, th = inputs.uniform_state(n, L, L, 21)
    m = oracle.Model(n=n, lx=L, ly=L, v=0.0, eta=eta, gamma=0.0, dt=dt, omega=om,
                     model=oracle.LANGEVIN, seed=4)
    _, _, t1, _, _, _ = oracle.step(m, x, y, th, 0)
    inc = _wrap(t1 - th - om * dt)
    assert stats.kstest(inc / (eta * np.sqrt(dt)), "norm").pvalue > 1e-4
    _, _, tT, _ = oracle.run(m, x, y, th, 0, T)
    c = np.cos(tT - th - om * dt * T)
    expect = np.exp(-eta**2 * dt * T / 2)
    assert abs(c.mean() - expect) < 5 * c.std() / np.sqrt(n)


@pytest.mark.parametrize("weight,order,c", [(0, 1, 1.0), (1, 1, 2.0), (0, 2, 1.0)])
def test_langevin_pair_relaxation_closed_form(oracle, weight, order, c):
    """Two particles, v = eta = 0: Delta = theta_1 - theta_2 obeys
    dDelta/dt = -c Gamma sin(o Delta) with c = 2 h(1) (h = 1/(1+n): c = 1;
    h = 1: c = 2), so tan(o Delta / 2) = tan(o Delta_0 / 2) exp(-o c Gamma t).
    Euler-Maruyama error is O(dt)."""
    g, dt, T = 1.3, 1e-3, 800
    m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, eta=0.0, gamma=g, dt=dt,
                     model=oracle.LANGEVIN, weight=weight, order=order)
    d0 = 1.2 if order == 1 else 0.6
    x, y, th = np.array([5.0, 5.5]), np.array([5.0, 5.0]), np.array([d0 / 2, -d0 / 2])
    _, _, tT, _ = oracle.run(m, x, y, th, 0, T)
    d = tT[0] - tT[1]
    expect = 2.0 / order * math.atan(math.tan(order * d0 / 2) * math.exp(-order * c * g * dt * T))
    assert abs(d - expect) < 5 * dt
    assert abs(d - d0) > 0.1  # it did relax


# ------------------------------------------------------ boundary rules ------

@pytest.mark.parametrize("wall", ["x0", "xL", "y0", "yL"])
def test_reflecting_single_particle(oracle, wall):
    """Re-entry at a reflecting wall: x -> -x or 2L - x with theta -> pi - theta;
    y -> -y or 2L - y with theta -> -theta (Sec. 2.4)."""
    L = 6.0
    pos = {"x0": (0.6, 3.0, np.pi), "xL": (L - 0.6, 3.0, 0.0),
           "y0": (3.0, 0.6, -np.pi / 2), "yL": (3.0, L - 0.6, np.pi / 2)}[wall]
    m = oracle.Model(n=1, lx=L, ly=L, v=1.0, eta=0.0, bx=1, by=1)
    xo, yo, to, nb, _, _ = oracle.step(m, np.array([pos[0]]), np.array([pos[1]]), np.array([pos[2]]), 0)
    assert nb[0] == 0
    if wall == "x0":
        assert abs(xo[0] - 0.4) < 1e-12 and abs(_wrap(to[0] - 0.0)) < 1e-12
    elif wall == "xL":
        assert abs(xo[0] - (L - 0.4)) < 1e-12 and abs(_wrap(to[0] - np.pi)) < 1e-12
    elif wall == "y0":
        assert abs(yo[0] - 0.4) < 1e-12 and abs(_wrap(to[0] - np.pi / 2)) < 1e-12
    else:
        assert abs(yo[0] - (L - 0.4)) < 1e-12 and abs(_wrap(to[0] + np.pi / 2)) < 1e-12


@pytest.mark.parametrize("model,bx,by", [(0, 1, 0), (0, 0, 1), (1, 1, 1), (1, 1, 0), (1, 0, 1)])
def test_reflecting_equals_mirror_extended_periodic_system(oracle, model, bx, by):
    """At eta = 0 the reflecting system on [0,L]^2 evolves exactly like the
    periodic system on the doubled box made of mirror copies (x, y, theta),
    (2L-x, y, pi-theta), (x, 2L-y, -theta), (2L-x, 2L-y, theta+pi),
    restricted to the first copy.  Pins the image rule, the own-image reading
    and the re-entry rule together.  The VM is checked with one reflecting
    axis (in a doubly reflecting corner its sum cancels exactly, see
    test_vm_reflecting_corner_cancellation); the NVM is left out because a lone
    wall particle takes exactly theta = 0 or +-pi/2, where sign(cos(theta_i -
    theta_j)) of Eq. (collision_NVM) is discontinuous and rounding decides."""
    lx, ly, n, T = 9.0, 8.0, 160, 12
    x, y, th = inputs.uniform_state(n, lx, ly, 30 + model)
    x[:10] = np.linspace(0.05, 0.9, 10)
    v, dt = (0.5, 1.0) if model != 1 else (1.0, 0.05)
    common = dict(v=v, eta=0.0, dt=dt, gamma=1.0, model=model)
    ref = oracle.Model(n=n, lx=lx, ly=ly, bx=bx, by=by, **common)
    xr, yr, tr, _ = oracle.run(ref, x, y, th, 0, T)
    xe, ye, te = _mirror_extension(x, y, th, lx, ly, bx, by)
    ext = oracle.Model(n=xe.size, lx=lx * (2 if bx else 1), ly=ly * (2 if by else 1), **common)
    xq, yq, tq, _ = oracle.run(ext, xe, ye, te, 0, T)
    # each original particle's copy that sits in the first quadrant
    k = np.arange(xe.size) % n
    inq = (xq <= lx) & (yq <= ly)
    for i in range(n):
        c = np.nonzero((k == i) & inq)[0]
        assert c.size == 1
        j = c[0]
        assert abs(xq[j] - xr[i]) < 1e-9 and abs(yq[j] - yr[i]) < 1e-9
        assert abs(_wrap(tq[j] - tr[i])) < 1e-9


def test_vm_reflecting_corner_cancellation(oracle):
    """With both walls reflecting, a particle within R/2 of a corner sees its
    three own mirror images, e^{i th} + e^{i(pi-th)} + e^{-i th} + e^{i(th+pi)} = 0:
    the VM sum vanishes and its argument is undefined (a property of the image
    rule of Sec. 2.4, reported as ill-conditioned in the parity tests)."""
    m = oracle.Model(n=1, lx=6.0, ly=6.0, v=0.0, eta=0.0, bx=1, by=1)
    _, _, _, nb, sm, _ = oracle.step(m, np.array([0.2]), np.array([0.3]), np.array([0.7]), 0)
    assert nb[0] == 3
    assert sm[0] < 1e-14


def test_periodic_translation_invariance(oracle):
    """Shifting every particle by an arbitrary vector (mod L) commutes with the
    periodic dynamics (the noise is keyed on particle id, not position)."""
    n, L, T = 600, 16.0, 6
    x, y, th = inputs.uniform_state(n, L, L, 41)
    m = oracle.Model(n=n, lx=L, ly=L, eta=0.4, seed=9)
    a, b = 5.3172, 11.0041
    x1, y1, t1, _ = oracle.run(m, x, y, th, 0, T)
    x2, y2, t2, _ = oracle.run(m, np.mod(x + a, L), np.mod(y + b, L), th, 0, T)
    dx = np.mod(x2 - a - x1 + L / 2, L) - L / 2
    dy = np.mod(y2 - b - y1 + L / 2, L) - L / 2
    assert np.abs(dx).max() < 1e-9 and np.abs(dy).max() < 1e-9
    assert np.abs(_wrap(t2 - t1)).max() < 1e-9


def test_permutation_invariance_without_noise(oracle):
    """At eta = 0 relabelling the particles only relabels the trajectory."""
    n, L, T = 500, 14.0, 8
    x, y, th = inputs.uniform_state(n, L, L, 43)
    perm = np.random.default_rng(1).permutation(n)
    m = oracle.Model(n=n, lx=L, ly=L, eta=0.0)
    x1, y1, t1, _ = oracle.run(m, x, y, th, 0, T)
    x2, y2, t2, _ = oracle.run(m, x[perm], y[perm], th[perm], 0, T)
    assert np.abs(x2 - x1[perm]).max() < 1e-10 and np.abs(_wrap(t2 - t1[perm])).max() < 1e-10


# ----------------------------------------------------------- observables ----

def test_polar_and_nematic_closed_forms(oracle):
    """p = |mean e^{i theta}| and q = |mean e^{2 i theta}| (Sec. 3.4)."""
    assert abs(oracle.polar(np.full(7, 0.4)) - 1.0) < 1e-15
    assert abs(oracle.polar(np.array([0.3, 0.3 + np.pi]))) < 1e-15
    assert abs(oracle.nematic(np.array([0.3, 0.3 + np.pi])) - 1.0) < 1e-15
    th = np.array([0.0, np.pi / 2])
    assert abs(oracle.polar(th) - np.sqrt(2) / 2) < 1e-15


def test_cell_step_equals_brute_force_neighbour_sums(oracle):
    """The cell-list step gathers the same neighbours (with image angles) as the
    brute-force definition: recompute the VM sum from brute-force lists."""
    n, L = 250, 9.0
    for bx, by in [(0, 0), (1, 1), (1, 0)]:
        x, y, th = inputs.uniform_state(n, L, L, 50 + bx + by)
        m = oracle.Model(n=n, lx=L, ly=L, bx=bx, by=by, eta=0.0, v=0.0)
        _, _, to, nb, sm, _ = oracle.step(m, x, y, th, 0)
        for i in range(0, n, 7):
            cnt, js, imgs = oracle.neighbours_brute(m, x, y, i)
            s = np.exp(1j * th[i])
            for j, im in zip(js, imgs):
                ix, iy = im % 3 - 1, im // 3 - 1
                t = th[j]
                if ix and bx:
                    t = np.pi - t
                if iy and by:
                    t = -t
                s += np.exp(1j * t)
            assert cnt == nb[i]
            assert abs(abs(s) - sm[i]) < 1e-12
            assert abs(_wrap(np.angle(s) - to[i])) < 1e-12


# ------------------------------------------- metric-free neighbourhoods -----

@pytest.mark.parametrize("k", [1, 6, 17])
def test_knn_periodic_matches_kdtree(oracle, k):
    """Metric-free neighbourhood (Sec. 2.3) in a periodic box = the k nearest
    other particles returned by scipy's periodic k-d tree."""
    lx, ly, n = 40.0, 25.0, 1500
    x, y, _ = inputs.uniform_state(n, lx, ly, 30 + k)
    m = oracle.Model(n=n, lx=lx, ly=ly, kn=k)
    tree = cKDTree(np.c_[x, y], boxsize=[lx, ly])
    for i in np.random.default_rng(k).choice(n, 150, replace=False):
        d_ref, j_ref = tree.query([x[i], y[i]], k=k + 1)
        j, img, d = oracle.knn(m, x, y, int(i), k)
        assert j_ref[0] == i and (j == j_ref[1:]).all()
        assert np.allclose(d, d_ref[1:], rtol=0, atol=1e-12)


@pytest.mark.parametrize("bx,by", [(1, 0), (0, 1), (1, 1)])
def test_knn_reflecting_matches_mirror_extension(oracle, bx, by):
    """Reflecting walls with image particles (Sec. 2.4) in the metric-free
    neighbourhood = the k nearest in the periodic doubled box of mirror
    copies (k-d tree); own mirror images take part like any other image."""
    lx, ly, n, k = 14.0, 11.0, 500, 7
    x, y, th = inputs.uniform_state(n, lx, ly, 40 + bx + 2 * by)
    x[:15] = np.linspace(0.02, 0.6, 15)
    y[15:30] = ly - np.linspace(0.02, 0.6, 15)
    m = oracle.Model(n=n, lx=lx, ly=ly, bx=bx, by=by, kn=k)
    xe, ye, _ = _mirror_extension(x, y, th, lx, ly, bx, by)
    box = [lx * (2 if bx else 1), ly * (2 if by else 1)]
    tree = cKDTree(np.c_[xe, ye], boxsize=box)
    ncopy = xe.size // n
    flips = [(0, 0), (1, 0), (0, 1), (1, 1)] if (bx and by) else ([(0, 0), (1, 0)] if bx else [(0, 0), (0, 1)])
    for i in list(range(30)) + list(np.random.default_rng(3).choice(n, 60, replace=False)):
        d_ref, e_ref = tree.query([x[i], y[i]], k=k + 1)
        assert e_ref[0] == i
        j, img, d = oracle.knn(m, x, y, int(i), k)
        assert np.allclose(d, d_ref[1:], rtol=0, atol=1e-12)
        # image code (ix+1) + 3 (iy+1): a nonzero ix is a mirror image only at a reflecting axis
        got = sorted((int(jj), int(bx and c % 3 != 1), int(by and c // 3 != 1)) for jj, c in zip(j, img))
        ref = sorted((int(e % n),) + flips[int(e // n)] for e in e_ref[1:])
        assert got == ref and ncopy == len(flips)


def test_mfvm_all_neighbours_reach_the_global_mean(oracle):
    """k >= N-1: every particle's neighbourhood is all the others, so at
    eta = omega = 0 every particle takes arg sum_j e^{i theta_j} (Eq. collision_VM)."""
    for k in (11, 30):
        m = oracle.Model(n=12, lx=20.0, ly=20.0, v=0.3, eta=0.0, kn=k)
        x, y, th = inputs.uniform_state(12, 20.0, 20.0, 5)
        xo, yo, to, nb, _, _ = oracle.step(m, x, y, th, 0)
        mean = math.atan2(np.sin(th).sum(), np.cos(th).sum())
        assert np.abs(_wrap(to - mean)).max() < 1e-12
        assert (nb == 11).all()
        assert np.allclose(np.mod(x + 0.3 * math.cos(mean), 20.0), xo, atol=1e-12)


def test_mfvm_pair_with_noise_closed_form(oracle):
    """N = 2, k = 1: each particle's neighbour is the other one wherever it is;
    theta' = arg(e^{i theta_i} + e^{i theta_j}) + omega + eta pi (2u - 1)."""
    m = oracle.Model(n=2, lx=30.0, ly=30.0, v=0.0, eta=0.3, omega=0.1, kn=1, seed=9)
    x, y, th = np.array([3.0, 25.0]), np.array([4.0, 17.0]), np.array([0.4, 2.9])
    _, _, to, nb, _, _ = oracle.step(m, x, y, th, 7)
    for i in range(2):
        u = oracle.u01(int(oracle.draw(m, i, 7, 0)[0]))
        e = math.atan2(math.sin(th[0]) + math.sin(th[1]), math.cos(th[0]) + math.cos(th[1]))
        assert abs(_wrap(to[i] - (e + 0.1 + 0.3 * math.pi * (2 * u - 1)))) < 1e-12
    assert (nb == 1).all()


def test_mfnvm_anti_aligned_pair(oracle):
    """mfNVM (Eq. collision_NVM with the k = 1 neighbourhood): a partner more
    than pi/2 away enters reversed, so the pair keeps its axis."""
    m = oracle.Model(n=2, lx=30.0, ly=30.0, v=0.0, eta=0.0, model=oracle.NVM, kn=1)
    a, b = 0.2, 0.2 + np.pi - 0.4
    _, _, to, _, _, _ = oracle.step(m, np.array([5.0, 20.0]), np.array([5.0, 9.0]), np.array([a, b]), 0)
    ea = math.atan2(math.sin(a) + math.sin(b + np.pi), math.cos(a) + math.cos(b + np.pi))
    assert abs(_wrap(to[0] - ea)) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_mfl_pair_relaxation_uses_h_equal_one(oracle, order):
    """mfL (Sec. 2.3): h = 1 whatever the weight setting, so a k = 1 pair at
    v = eta = 0 relaxes as tan(o Delta / 2) = tan(o Delta_0 / 2) exp(-2 o Gamma t)."""
    g, dt, T = 0.9, 1e-3, 700
    m = oracle.Model(n=2, lx=30.0, ly=30.0, v=0.0, eta=0.0, gamma=g, dt=dt, model=oracle.LANGEVIN,
                     weight=0, order=order, kn=1)
    d0 = 1.1 if order == 1 else 0.5
    x, y, th = np.array([2.0, 21.0]), np.array([3.0, 14.0]), np.array([d0 / 2, -d0 / 2])
    _, _, tT, _ = oracle.run(m, x, y, th, 0, T)
    expect = 2.0 / order * math.atan(math.tan(order * d0 / 2) * math.exp(-order * 2 * g * dt * T))
    assert abs((tT[0] - tT[1]) - expect) < 5 * dt


def test_knn_band_flags_near_ties(oracle):
    """The ambiguity flag marks particles whose k-th and (k+1)-th nearest
    candidates are closer than `band` to each other."""
    m = oracle.Model(n=3, lx=20.0, ly=20.0, v=0.0, eta=0.0, kn=1)
    x, y, th = np.array([10.0, 11.0, 9.0 + 1e-7]), np.array([10.0, 10.0, 10.0]), np.zeros(3)
    amb = oracle.step(m, x, y, th, 0, band=1e-5)[5]
    assert amb[0] == 1 and amb[1] == 0


# ------------------------------------------------------------- species -----

def test_species_blocks_of_ids(oracle):
    """Species are consecutive blocks of particle ids (Sec. 2.5 gives N as a list)."""
    m = oracle.Model(n=10, lx=10.0, ly=10.0, species_n=(3, 0, 7))
    p = m.c()
    got = [oracle.lib().orc_species_of(ctypes.byref(p), i) for i in range(10)]
    assert got == [0, 0, 0, 2, 2, 2, 2, 2, 2, 2]


def test_species_isolated_particles_closed_form(oracle):
    """Three isolated particles of three species (VM, Sec. 2.1 + 2.5): each
    turns by its own omega_s + eta_s pi (2u - 1) and moves by its own v_s."""
    v, eta, om = (0.1, 0.3, 0.5), (0.0, 0.2, 0.6), (0.05, -0.3, 0.0)
    m = oracle.Model(n=3, lx=30.0, ly=30.0, species_n=(1, 1, 1), species_v=v, species_eta=eta,
                     species_omega=om, seed=3)
    x, y, th = np.array([5.0, 15.0, 25.0]), np.array([5.0, 15.0, 25.0]), np.array([0.3, -1.0, 2.0])
    xo, yo, to, _, _, _ = oracle.step(m, x, y, th, 4)
    for i in range(3):
        u = oracle.u01(int(oracle.draw(m, i, 4, 0)[0]))
        t = th[i] + om[i] + eta[i] * math.pi * (2 * u - 1)
        assert abs(_wrap(to[i] - t)) < 1e-12
        assert abs(xo[i] - (x[i] + v[i] * math.cos(t))) < 1e-12
        assert abs(yo[i] - (y[i] + v[i] * math.sin(t))) < 1e-12


def test_species_ordered_mixture_translates_at_own_speeds(oracle):
    """eta = omega = 0, every theta equal: the VM keeps the common angle, and
    each species translates rigidly with its own speed."""
    n, L, t0 = 900, 20.0, 0.7
    x, y, _ = inputs.uniform_state(n, L, L, 8)
    th = np.full(n, t0)
    m = oracle.Model(n=n, lx=L, ly=L, eta=0.0, species_n=(300, 600), species_v=(0.2, 0.7))
    xT, yT, tT, _ = oracle.run(m, x, y, th, 0, 5)
    assert np.abs(_wrap(tT - t0)).max() < 1e-12
    v = np.where(np.arange(n) < 300, 0.2, 0.7)
    assert np.allclose(xT, np.mod(x + 5 * v * math.cos(t0), L), atol=1e-9)
    assert np.allclose(yT, np.mod(y + 5 * v * math.sin(t0), L), atol=1e-9)


def test_species_langevin_pair_nonreciprocal_coupling(oracle):
    """Langevin A-B pair, v = eta = 0, h = 1/(1+n) = 1/2 (Eq. Langevin_dynamics
    with Gamma_{s_i s_j}): each Euler-Maruyama step conserves
    Gamma_BA theta_A + Gamma_AB theta_B exactly, and Delta = theta_A - theta_B
    relaxes as tan(Delta/2) = tan(Delta_0/2) exp(-(Gamma_AB + Gamma_BA) t / 2)."""
    gab, gba, dt, T = 1.6, 0.4, 1e-3, 900
    G = ((0.0, gab), (gba, 0.0))
    m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, eta=0.0, dt=dt, model=oracle.LANGEVIN,
                     species_n=(1, 1), species_v=(0.0, 0.0), species_eta=(0.0, 0.0),
                     species_omega=(0.0, 0.0), species_gamma=G)
    x, y, th = np.array([5.0, 5.5]), np.array([5.0, 5.0]), np.array([0.6, -0.5])
    inv0 = gba * th[0] + gab * th[1]
    xs, ys, ts = x, y, th
    for t in range(5):
        xs, ys, ts, _, _, _ = oracle.step(m, xs, ys, ts, t)
        assert abs(gba * ts[0] + gab * ts[1] - inv0) < 1e-14
    _, _, tT, _ = oracle.run(m, x, y, th, 0, T)
    d0 = th[0] - th[1]
    expect = 2 * math.atan(math.tan(d0 / 2) * math.exp(-(gab + gba) / 2 * dt * T))
    assert abs((tT[0] - tT[1]) - expect) < 5 * dt
    assert abs(gba * tT[0] + gab * tT[1] - inv0) < 1e-12


def test_species_one_way_coupling_leaves_the_leader_free(oracle):
    """Gamma_AB = 0: species A ignores B, so at eta = 0 it just rotates with
    omega_A; B (Gamma_BA > 0) turns towards A (metric-free k = 1 as well)."""
    for kn in (0, 1):
        m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, dt=0.01, model=oracle.LANGEVIN, kn=kn,
                         species_n=(1, 1), species_v=(0.0, 0.0), species_eta=(0.0, 0.0),
                         species_omega=(0.3, 0.0), species_gamma=((0.0, 0.0), (2.0, 0.0)))
        x, y, th = np.array([5.0, 5.5]), np.array([5.0, 5.0]), np.array([0.2, 1.5])
        _, _, tT, _ = oracle.run(m, x, y, th, 0, 100)
        assert abs(_wrap(tT[0] - (0.2 + 0.3 * 0.01 * 100))) < 1e-12
        assert abs(_wrap(tT[1] - tT[0])) < abs(_wrap(th[1] - th[0])) - 0.3


def test_species_identical_parameters_reduce_to_one_species(oracle):
    """Splitting one species into identical ones changes nothing (Langevin,
    with the coupling moved inside the sum: equal up to rounding)."""
    n, L = 700, 15.0
    x, y, th = inputs.uniform_state(n, L, L, 12)
    kw = dict(n=n, lx=L, ly=L, v=0.3, eta=0.2, omega=0.1, gamma=1.3, dt=0.05, model=oracle.LANGEVIN)
    a = oracle.step(oracle.Model(**kw), x, y, th, 2)
    G = ((1.3, 1.3), (1.3, 1.3))
    b = oracle.step(oracle.Model(**kw, species_n=(200, 500), species_v=(0.3, 0.3), species_eta=(0.2, 0.2),
                                 species_omega=(0.1, 0.1), species_gamma=G), x, y, th, 2)
    for u, w in zip(a[:3], b[:3]):
        assert np.allclose(u, w, rtol=0, atol=1e-12)


# ------------------------------------------------ tabulated weight h(n) -----

def test_weight_table_reduces_to_the_built_in_weights(oracle):
    """A table h(n) = 1/(1+n) or h = 1 (Sec. 4's weight_function, sampled at
    n = 0 .. len-1) gives the built-in weights."""
    n, L = 800, 16.0
    x, y, th = inputs.uniform_state(n, L, L, 14)
    kw = dict(n=n, lx=L, ly=L, v=0.3, eta=0.2, gamma=1.4, dt=0.05, model=oracle.LANGEVIN)
    for weight, table in ((0, tuple(1.0 / (1.0 + k) for k in range(64))), (1, (1.0,) * 3)):
        a = oracle.step(oracle.Model(**kw, weight=weight), x, y, th, 1)
        b = oracle.step(oracle.Model(**kw, weight=1 - weight, weight_table=table), x, y, th, 1)
        for u, w in zip(a[:3], b[:3]):
            assert np.array_equal(u, w)


def test_weight_table_pair_rate_and_clamp(oracle):
    """A pair at v = eta = 0 relaxes at rate 2 h(1) Gamma (tan(Delta/2) law); a
    particle with more neighbours than the table covers uses its last entry."""
    g, dt, T, c = 1.1, 1e-3, 600, 0.37
    m = oracle.Model(n=2, lx=10.0, ly=10.0, v=0.0, eta=0.0, gamma=g, dt=dt, model=oracle.LANGEVIN,
                     weight_table=(5.0, c))
    d0 = 1.0
    _, _, tT, _ = oracle.run(m, np.array([5.0, 5.5]), np.array([5.0, 5.0]), np.array([d0 / 2, -d0 / 2]), 0, T)
    expect = 2 * math.atan(math.tan(d0 / 2) * math.exp(-2 * c * g * dt * T))
    assert abs((tT[0] - tT[1]) - expect) < 5 * dt
    # four particles within R of each other: n = 3 > len - 1 = 1 -> h = c
    m4 = oracle.Model(n=4, lx=10.0, ly=10.0, v=0.0, eta=0.0, gamma=g, dt=dt, model=oracle.LANGEVIN,
                      weight_table=(5.0, c))
    x = np.array([5.0, 5.3, 5.0, 5.3]); y = np.array([5.0, 5.0, 5.3, 5.3]); th = np.array([0.1, 0.7, -0.4, 1.2])
    _, _, t1, nb, _, _ = oracle.step(m4, x, y, th, 0)
    assert (nb == 3).all()
    for i in range(4):
        s = sum(math.sin(th[j] - th[i]) for j in range(4) if j != i)
        assert abs(_wrap(t1[i] - (th[i] + dt * g * c * s))) < 1e-14
