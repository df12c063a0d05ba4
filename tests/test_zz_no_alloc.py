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

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _fields_both_ways(h, p, nb, stream):
    ref = torch.zeros(3 * nb * nb, dtype=torch.float32, device="cuda")
    A.aap_coarse_grain(h, nb, nb, ref.data_ptr())
    A.aap_sync(h)
    x, y, th = A.aap_get_state(h, p.n)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    td = torch.from_numpy(th).cuda()
    out = torch.full((3 * nb * nb,), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    A.aap_coarse_grain_noalloc(xd.data_ptr(), yd.data_ptr(), td.data_ptr(), p.n, p.lx, p.ly, nb, nb,
                               out.data_ptr(), stream)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_coarse_grain_matches_two_calls_in_a_row(lib):
    p = A.aap_params_default(n=1 << 17, lx=256.0, ly=256.0, eta=0.4, seed=21)
    h = A.aap_create(p)
    try:
        for k in range(2):                       # two calls, different states
            A.aap_step(h, 7 + k)
            ref, got = _fields_both_ways(h, p, 64, 0)
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
        ref, got = _fields_both_ways(h, p, 97, 0)
        assert np.array_equal(got, ref)
    finally:
        A.aap_destroy(h)


def test_noalloc_rejects_too_many_bins(lib):
    with pytest.raises(A.AapError) as e:
        A.aap_coarse_grain_noalloc(0, 0, 0, 0, 10.0, 10.0, 512, 512, 1, 0)
    assert e.value.code == A.AAP_EINVAL
    assert "exceeds" in str(e.value)
