"""Failure detection without a GPU fault: allocation failures injected on the
host (aap_test_fail_alloc_after) at every allocation of aap_create must return
AAP_ENOMEM, release everything the call had taken, and leave the library
usable; a failed allocation inside a call on a live handle leaves the handle
usable.  The pipelined step kernel's bounded waits are made to run out by a
withheld tile (aap_test_pipe_wait): the kernel ends with AAP_ETIMEOUT and the
context stays usable."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from tests.gpu_helpers import params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("kw", [dict(), dict(kn=6), dict(model=A.AAP_LANGEVIN, dt=0.05, bx=1)])
def test_create_fails_cleanly_at_every_allocation(lib, kw):
    p = params(n=60000, lx=170.0, ly=170.0, seed=5, **kw)
    h = A.aap_create(p)                      # warm the context and the kernels
    A.aap_step(h, 2)
    A.aap_destroy(h)
    free0 = _free()
    failures = 0
    try:
        for k in range(200):
            A.aap_test_fail_alloc_after(k)
            try:
                h = A.aap_create(p)
            except A.AapError as e:
                assert e.code == A.AAP_ENOMEM and "injected" in str(e)
                failures += 1
                assert abs(_free() - free0) < (8 << 20), f"allocation {k}: memory not released"
                continue
            break
    finally:
        A.aap_test_fail_alloc_after(-1)
    assert failures >= 10                    # every allocation of the handle was exercised
    A.aap_step(h, 3)
    assert np.isfinite(A.aap_observe(h).phi)
    A.aap_destroy(h)
    assert abs(_free() - free0) < (8 << 20)


def test_failed_allocation_inside_a_call_keeps_the_handle(lib):
    p = params(n=40000, lx=140.0, ly=140.0, seed=6)
    h = A.aap_create(p)
    try:
        A.aap_step(h, 4)
        A.aap_test_fail_alloc_after(0)
        with pytest.raises(A.AapError) as e:
            A.aap_phi_trace(h, 16)           # needs a trace buffer
        assert e.value.code == A.AAP_ENOMEM
        A.aap_test_fail_alloc_after(0)
        with pytest.raises(A.AapError) as e:
            A.aap_step_neighbours(h, p.n)    # needs a neighbour buffer
        assert e.value.code == A.AAP_ENOMEM
        A.aap_test_fail_alloc_after(-1)
        phi = A.aap_phi_trace(h, 16)
        assert phi.shape == (17,) and np.isfinite(phi).all()
        assert A.aap_step_neighbours(h, p.n).shape == (p.n,)
    finally:
        A.aap_test_fail_alloc_after(-1)
        A.aap_destroy(h)


def test_pipeline_wait_runs_out_and_reports(lib):
    """The pipelined step kernel's hand-offs are bounded mbarrier waits.  With
    the bound shortened to 2e7 SM cycles and every block's copy warp
    withholding its first tile (a fill that never arrives), the sort and update
    warps behind it give up, the kernel sets its timeout bit and ends, later
    steps of the handle return at once, and the handle reports AAP_ETIMEOUT at
    its next synchronising call.  The context stays usable: afterwards a fresh
    pipelined handle and a whole-block one agree bit for bit."""
    p = params(n=30000, lx=122.0, ly=122.0, eta=0.35, v=0.5, seed=19, threads=1024)
    A.aap_test_pipe_wait(20_000_000, 1)
    try:
        h = A.aap_create(p)
        try:
            assert A.aap_get_layout(h).threads == 1024
            A.aap_step(h, 3)
            with pytest.raises(A.AapError) as e:
                A.aap_observe(h)
            assert e.value.code == A.AAP_ETIMEOUT
        finally:
            A.aap_destroy(h)
    finally:
        A.aap_test_pipe_wait(0, 0)
    q = params(n=30000, lx=122.0, ly=122.0, eta=0.35, v=0.5, seed=19, threads=512)
    h1, h2 = A.aap_create(p), A.aap_create(q)
    try:
        for h in (h1, h2):
            A.aap_step(h, 12)
        for u, v in zip(A.aap_get_state(h1, p.n), A.aap_get_state(h2, p.n)):
            assert np.array_equal(u, v)
    finally:
        A.aap_destroy(h1)
        A.aap_destroy(h2)
