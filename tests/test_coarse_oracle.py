"""Pins of the coarse-graining oracle (oracle/coarse.py) against facts that
do not come from it: a hand-worked fixture, conservation of the particle
number and of sum_i e^{i theta_i} (so the fields' polar order parameter is
the particles' one, Sec. 3.4), counting by explicit bin intervals, and the
shift of the fields under a translation by one bin (which separates the x
and y axes on a grid with nbx != nby)."""
import numpy as np
import pytest

from oracle import coarse as CG


def test_hand_worked_fixture():
    """Box 10 x 6, 5 x 3 bins of 2 x 2 (area 4).  Worked by hand:
    (0.5, 0.5, 0)       -> bin (y 0, x 0)
    (3.9, 0.1, pi/2)    -> bin (0, 1)    3.9 / 2 = 1.95
    (9.99, 5.99, pi)    -> bin (2, 4)
    (10.0, 6.0, 0)      -> bin (2, 4)    x = lx, y = ly belong to the last bins
    (4.0, 2.0, -pi/2)   -> bin (1, 2)    on the lower-left edge of bin (1, 2)."""
    x = np.array([0.5, 3.9, 9.99, 10.0, 4.0])
    y = np.array([0.5, 0.1, 5.99, 6.0, 2.0])
    th = np.array([0.0, np.pi / 2, np.pi, 0.0, -np.pi / 2])
    f = CG.coarse_grain(x, y, th, 10.0, 6.0, 5, 3)
    rho = np.zeros((3, 5))
    rho[0, 0] = rho[0, 1] = rho[1, 2] = 0.25
    rho[2, 4] = 0.5
    px = np.zeros((3, 5))
    px[0, 0] = 0.25                       # cos 0; bin (2, 4): cos pi + cos 0 = 0
    py = np.zeros((3, 5))
    py[0, 1] = 0.25
    py[1, 2] = -0.25
    assert np.array_equal(f[0], rho)
    assert np.allclose(f[1], px, atol=1e-15)
    assert np.allclose(f[2], py, atol=1e-15)
    assert np.array_equal(CG.counts(x, y, 10.0, 6.0, 5, 3), (rho * 4).astype(np.int64))


def _state(n, lx, ly, seed):
    g = np.random.default_rng(seed)
    return g.uniform(0, lx, n), g.uniform(0, ly, n), g.uniform(-np.pi, np.pi, n)


@pytest.mark.parametrize("nbx,nby", [(1, 1), (7, 3), (64, 64), (97, 64)])
def test_conservation_and_order_parameter(oracle, nbx, nby):
    lx, ly = 123.0, 77.5
    x, y, th = _state(5000, lx, ly, nbx * 100 + nby)
    f = CG.coarse_grain(x, y, th, lx, ly, nbx, nby)
    area = (lx / nbx) * (ly / nby)
    assert np.round(f[0] * area).sum() == 5000
    s = complex(np.cos(th).sum(), np.sin(th).sum())
    assert abs(f[1].sum() * area - s.real) < 1e-9 and abs(f[2].sum() * area - s.imag) < 1e-9
    phi_fields = np.hypot(f[1].sum(), f[2].sum()) * area / 5000
    assert abs(phi_fields - oracle.polar(th)) < 1e-12
    if nbx == nby == 1:
        assert abs(f[0][0, 0] - 5000 / (lx * ly)) < 1e-12


def test_counts_by_explicit_intervals():
    """Count each bin by testing lo <= x < hi with lo, hi = k L / nb (a
    different formulation from the floor of a product)."""
    lx, ly, nbx, nby = 50.0, 30.0, 11, 6
    x, y, th = _state(400, lx, ly, 3)
    c = CG.counts(x, y, lx, ly, nbx, nby)
    for j in range(nby):
        for i in range(nbx):
            inside = ((x >= i * lx / nbx) & (x < (i + 1) * lx / nbx) &
                      (y >= j * ly / nby) & (y < (j + 1) * ly / nby))
            assert c[j, i] == inside.sum()


def test_translation_by_one_bin_shifts_the_fields():
    """Periodic box: moving every particle by one bin width along x rolls the
    fields by one column, along y by one row (nbx != nby, so a swapped axis
    or a transposed plane fails)."""
    lx, ly, nbx, nby = 40.0, 24.0, 8, 4
    wx, wy = lx / nbx, ly / nby
    g = np.random.default_rng(5)
    # positions well inside their bins, so the shifted products stay off the edges
    ix = g.integers(0, nbx, 300)
    iy = g.integers(0, nby, 300)
    x = (ix + g.uniform(0.1, 0.9, 300)) * wx
    y = (iy + g.uniform(0.1, 0.9, 300)) * wy
    th = g.uniform(-np.pi, np.pi, 300)
    f = CG.coarse_grain(x, y, th, lx, ly, nbx, nby)
    fx = CG.coarse_grain(np.mod(x + wx, lx), y, th, lx, ly, nbx, nby)
    fy = CG.coarse_grain(x, np.mod(y + wy, ly), th, lx, ly, nbx, nby)
    assert np.allclose(fx, np.roll(f, 1, axis=2), atol=1e-12)
    assert np.allclose(fy, np.roll(f, 1, axis=1), atol=1e-12)
    assert not np.allclose(fx, np.roll(f, 1, axis=1), atol=1e-12)
