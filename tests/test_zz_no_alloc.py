"""aap_coarse_grain_noalloc: coarse-graining for callers that cannot allocate
device memory (their memory belongs to a pool or arena, or they must not call
cudaMalloc, for instance while a stream is being captured).  It bins
caller-owned device arrays with a fixed internal scratch instead of library
allocations; its fields must equal those of aap_coarse_grain on the same
state.  Collected last on purpose (file name), so that a run stopping at the
first failure has already run everything else."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from oracle import coarse as CG

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _fields_both_ways(h, p, nb, stream, nby=None):
    nby = nb if nby is None else nby
    ref = torch.zeros(3 * nb * nby, dtype=torch.float32, device="cuda")
    A.aap_coarse_grain(h, nb, nby, ref.data_ptr())
    A.aap_sync(h)
    x, y, th = A.aap_get_state(h, p.n)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    td = torch.from_numpy(th).cuda()
    out = torch.full((3 * nb * nby,), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    A.aap_coarse_grain_noalloc(xd.data_ptr(), yd.data_ptr(), td.data_ptr(), p.n, p.lx, p.ly, nb, nby,
                               out.data_ptr(), stream)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy(), (x, y, th)


def _oracle_close(got, state, p, nbx, nby):
    """Counts equal to the oracle's, polarisation within FP32 rounding."""
    x, y, th = state
    f = got.reshape(3, nby, nbx).astype(np.float64)
    area = (p.lx / nbx) * (p.ly / nby)
    counts = CG.counts(x, y, p.lx, p.ly, nbx, nby)
    assert np.array_equal(np.round(f[0] * area), counts)
    ref = CG.coarse_grain(x, y, th, p.lx, p.ly, nbx, nby)
    assert np.all(np.abs(f[1:] - ref[1:]) * area < 1e-6 * (counts + 1.0))


def test_noalloc_coarse_grain_matches_two_calls_in_a_row(lib):
    p = A.aap_params_default(n=1 << 17, lx=256.0, ly=256.0, eta=0.4, seed=21)
    h = A.aap_create(p)
    try:
        for k in range(2):                       # two calls, different states
            A.aap_step(h, 7 + k)
            ref, got, state = _fields_both_ways(h, p, 64, 0)
            _oracle_close(got, state, p, 64, 64)
            area = (p.lx / 64) * (p.ly / 64)
            assert np.isfinite(got).all()
            # the coarse-grain tests' tolerance; the integer sums make it exact
            assert np.allclose(got, ref, rtol=1e-6, atol=1e-6)
            assert np.array_equal(got, ref)
            assert abs(got[: 64 * 64].sum() * area - p.n) < 1e-3
    finally:
        A.aap_destroy(h)


def test_noalloc_matches_on_odd_bin_widths(lib):
    """Bin widths that are not powers of two: both entry points bin each
    particle at floor(x nb / L) of its FP64 position and sum the same integers."""
    p = A.aap_params_default(n=90000, lx=300.0, ly=300.0, eta=0.4, seed=23)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 5)
        ref, got, state = _fields_both_ways(h, p, 97, 0)
        assert np.array_equal(got, ref)
        _oracle_close(got, state, p, 97, 97)
    finally:
        A.aap_destroy(h)


def test_noalloc_matches_on_a_rectangular_grid(lib):
    """nbx != nby: a swapped row / column index or a wrong plane stride would
    move sums between bins."""
    p = A.aap_params_default(n=60000, lx=240.0, ly=180.0, eta=0.4, seed=29)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 4)
        ref, got, state = _fields_both_ways(h, p, 97, 0, nby=64)
        assert np.array_equal(got, ref)
        _oracle_close(got, state, p, 97, 64)
    finally:
        A.aap_destroy(h)


def test_noalloc_empty_state_after_a_full_one(lib):
    """n = 0 right after a call that left sums in the shared array: the
    fields are all zero (the array is cleared at the start of each call)."""
    p = A.aap_params_default(n=20000, lx=100.0, ly=100.0, eta=0.4, seed=31)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 2)
        _, got, _ = _fields_both_ways(h, p, 16, 0)
        assert got[: 16 * 16].sum() > 0
        out = torch.full((3 * 16 * 16,), float("nan"), dtype=torch.float32, device="cuda")
        A.aap_coarse_grain_noalloc(0, 0, 0, 0, p.lx, p.ly, 16, 16, out.data_ptr(), 0)
        torch.cuda.synchronize()
        assert torch.equal(out, torch.zeros_like(out))
    finally:
        A.aap_destroy(h)


def test_noalloc_positions_outside_the_box(lib):
    """The documented clamping, worked by hand on a 10 x 10 box with 5 x 5
    bins: x < 0 and NaN go to the first column, x > lx to the last; a NaN
    orientation counts but adds no polarisation."""
    x = torch.tensor([-3.0, float("nan"), 12.0, 5.0], dtype=torch.float64, device="cuda")
    y = torch.tensor([1.0, 1.0, 1.0, 1e300], dtype=torch.float64, device="cuda")
    th = torch.tensor([0.0, 0.0, 0.0, float("nan")], dtype=torch.float32, device="cuda")
    out = torch.zeros(3 * 25, dtype=torch.float32, device="cuda")
    A.aap_coarse_grain_noalloc(x.data_ptr(), y.data_ptr(), th.data_ptr(), 4, 10.0, 10.0, 5, 5, out.data_ptr(), 0)
    torch.cuda.synchronize()
    f = out.cpu().numpy().reshape(3, 5, 5) * 4.0          # bin area 4: counts and sums
    want = np.zeros((5, 5))
    want[0, 0] = 2                                       # x = -3 and x = NaN, y = 1
    want[0, 4] = 1                                       # x = 12
    want[4, 2] = 1                                       # x = 5, y = 1e300
    assert np.array_equal(f[0], want)
    pol = np.zeros((5, 5))
    pol[0, 0] = 2.0
    pol[0, 4] = 1.0
    assert np.array_equal(f[1], pol) and np.array_equal(f[2], np.zeros((5, 5)))


def test_noalloc_rejects_a_non_finite_box(lib):
    for lx in (float("inf"), float("nan"), 0.0):
        with pytest.raises(A.AapError) as e:
            A.aap_coarse_grain_noalloc(0, 0, 0, 0, lx, 10.0, 4, 4, 1, 0)
        assert e.value.code == A.AAP_EINVAL


def test_noalloc_rejects_too_many_bins(lib):
    with pytest.raises(A.AapError) as e:
        A.aap_coarse_grain_noalloc(0, 0, 0, 0, 10.0, 10.0, 512, 512, 1, 0)
    assert e.value.code == A.AAP_EINVAL
    assert "exceeds" in str(e.value)


def test_noalloc_allocates_nothing_and_runs_in_a_captured_graph(lib):
    """The promise of the entry point: after a first call, a call changes the
    device's free memory by nothing, and it can be captured into a CUDA graph
    (where cudaMalloc is barred); the replayed graph gives the fields of a
    direct call."""
    p = A.aap_params_default(n=1 << 16, lx=181.0, ly=181.0, eta=0.4, seed=23)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 5)
        x, y, th = A.aap_get_state(h, p.n)
    finally:
        A.aap_destroy(h)
    xd, yd, td = (torch.from_numpy(v).cuda() for v in (x, y, th))
    nbx, nby = 90, 60
    direct = torch.zeros(3 * nbx * nby, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A.aap_coarse_grain_noalloc(xd.data_ptr(), yd.data_ptr(), td.data_ptr(), p.n, p.lx, p.ly, nbx, nby,
                                   direct.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(s):
        A.aap_coarse_grain_noalloc(xd.data_ptr(), yd.data_ptr(), td.data_ptr(), p.n, p.lx, p.ly, nbx, nby,
                                   direct.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    out = torch.full((3 * nbx * nby,), float("nan"), dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        A.aap_coarse_grain_noalloc(xd.data_ptr(), yd.data_ptr(), td.data_ptr(), p.n, p.lx, p.ly, nbx, nby,
                                   out.data_ptr(), s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, direct)
    _oracle_close(out.cpu().numpy(), (x, y, th), p, nbx, nby)
