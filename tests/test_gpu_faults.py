"""Failure detection without a GPU fault: allocation failures injected on the
host (aap_test_fail_alloc_after) at every allocation of aap_create must return
AAP_ENOMEM, release everything the call had taken, and leave the library
usable; a failed allocation inside a call on a live handle leaves the handle
usable."""
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
