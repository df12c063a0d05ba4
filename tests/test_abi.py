"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/aap.h declares; parameter validation fails
cleanly before any CUDA call."""
import os
import re

import pytest

import paper_2211_15630_gb300 as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(aap_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(A.EXPORTS) <= declared


def test_abi_version_and_defaults(lib):
    assert A.aap_abi_version() == 2
    p = A.aap_params_default()
    assert (p.n, p.lx, p.ly, p.r, p.v, p.eta, p.model, p.order, p.weight) == (
        1000, 32.0, 32.0, 1.0, 0.5, 0.4, A.AAP_VM, 1, A.AAP_H_INV_1PN)


@pytest.mark.parametrize("kw,frag", [
    (dict(lx=2.9), "3 cells"), (dict(n=-3), "n must"), (dict(v=1.2), "displacement"),
    (dict(model=9), "model"), (dict(eta=-0.1), "eta"), (dict(model=1, dt=-1.0), "dt"),
    (dict(order=0), "order"), (dict(weight=5), "weight"), (dict(threads=96), "threads"),
    (dict(tile_w=4), "tile_w"), (dict(capacity=0.5), "capacity"), (dict(r=float("inf")), "finite"),
    (dict(binnum_theta=513), "binnum"), (dict(binnum_neighbors=-1), "binnum"),
    (dict(kn=33), "kn"), (dict(kn=-1), "kn"), (dict(kn=4, n=1 << 28), "2^28"),
    (dict(kn=4, v=9.0), "quarter"), (dict(nspecies=9), "nspecies"),
    (dict(nspecies=2), "add up"), (dict(weight_len=129), "weight_len"),
])
def test_invalid_parameters(lib, kw, frag):
    with pytest.raises(A.AapError) as e:
        A.aap_create(A.aap_params_default(**kw))
    assert e.value.code == A.AAP_EINVAL
    assert frag in str(e.value)


def test_null_arguments(lib):
    import ctypes as C

    assert lib.aap_create(None, None, None) == A.AAP_EINVAL
    assert lib.aap_step(None, 1) == A.AAP_EINVAL
    assert lib.aap_observe(None, None) == A.AAP_EINVAL
    assert lib.aap_destroy(None) == A.AAP_OK
    assert b"NULL" in lib.aap_last_error() or lib.aap_last_error() == b""
    del C


def test_load_rejects_missing_and_foreign_files(lib, tmp_path):
    with pytest.raises(A.AapError) as e:
        A.aap_load(str(tmp_path / "absent.aap"))
    assert e.value.code == A.AAP_EIO
    junk = tmp_path / "junk.aap"
    junk.write_bytes(b"not a state file at all")
    with pytest.raises(A.AapError) as e:
        A.aap_load(str(junk))
    assert e.value.code == A.AAP_EIO and "not a saved state" in str(e.value)
    trunc = tmp_path / "trunc.aap"
    trunc.write_bytes(b"AAPSAVE1" + (1).to_bytes(4, "little"))
    with pytest.raises(A.AapError) as e:
        A.aap_load(str(trunc))
    assert e.value.code == A.AAP_EIO


def test_get_state_out_buffers_checked_before_the_call():
    """aap_get_state(h, n, out=...) rejects buffers of the wrong type or size
    before anything reaches the library (so no handle or GPU is needed)."""
    import numpy as np
    import paper_2211_15630_gb300 as A

    good = (np.zeros(4, np.float64), np.zeros(4, np.float64), np.zeros(4, np.float32))
    for bad in ((np.zeros(4, np.float32),) + good[1:],            # x not float64
                good[:2] + (np.zeros(4, np.float64),),            # theta not float32
                (np.zeros(3, np.float64),) + good[1:],            # too short
                (np.zeros(8, np.float64)[::2],) + good[1:]):      # not contiguous
        with pytest.raises(ValueError):
            A.aap_get_state(None, 4, out=bad)

