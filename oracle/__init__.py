"""FP64 CPU oracle for the aligning-active-particles update (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It wraps ``aap_oracle.c`` (plain C, FP64) through
ctypes; nothing here is shared with the CUDA library.  The functions follow
Kuersten, "Aligning Active Particles Py Package": Eq. (collision_VM),
Eq. (collision_NVM), Eq. (streaming), Eq. (Langevin_dynamics),
Eq. (metric_neighborhood), Sec. 2.4 (boundaries), Sec. 3.2 (cell lists),
Sec. 3.4 (order parameters).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

VM, LANGEVIN, NVM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile aap_oracle.c into oracle/liboracle.so with gcc (OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "aap_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
             _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``orc_params`` (aap_oracle.h)."""

    _fields_ = [
        ("n", C.c_int64), ("lx", C.c_double), ("ly", C.c_double), ("r", C.c_double),
        ("v", C.c_double), ("eta", C.c_double), ("omega", C.c_double),
        ("gamma", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
        ("model", C.c_int32), ("order", C.c_int32), ("weight", C.c_int32),
        ("bx", C.c_int32), ("by", C.c_int32), ("self_image", C.c_int32), ("kn", C.c_int32),
        ("nspecies", C.c_int32), ("pad_", C.c_int32), ("species_n", C.c_int64 * 8),
        ("species_v", C.c_double * 8), ("species_eta", C.c_double * 8),
        ("species_omega", C.c_double * 8), ("species_gamma", C.c_double * 64),
        ("weight_len", C.c_int32), ("pad2_", C.c_int32), ("weight_table", C.c_double * 128),
    ]


@dataclass
class Model:
    """Model parameters with the paper's names (Sec. 4 usage list)."""

    n: int
    lx: float
    ly: float
    r: float = 1.0
    v: float = 0.5
    eta: float = 0.4
    omega: float = 0.0
    gamma: float = 1.0
    dt: float = 1.0
    seed: int = 1
    model: int = VM
    order: int = 1
    weight: int = 0
    bx: int = 0
    by: int = 0
    self_image: int = 1
    kn: int = 0
    # species (Sec. 2.5): counts per species, then per-species v, eta, omega
    # and the coupling matrix gamma[a][b]; empty = one species
    species_n: tuple = ()
    species_v: tuple = ()
    species_eta: tuple = ()
    species_omega: tuple = ()
    species_gamma: tuple = ()
    # tabulated Langevin weight h(0), h(1), ... (Sec. 4); empty = `weight`
    weight_table: tuple = ()

    def c(self) -> Params:
        p = Params(self.n, self.lx, self.ly, self.r, self.v, self.eta, self.omega,
                   self.gamma, self.dt, self.seed, self.model, self.order, self.weight,
                   self.bx, self.by, self.self_image, self.kn)
        ns = len(self.species_n)
        p.nspecies = ns
        for s in range(ns):
            p.species_n[s] = int(self.species_n[s])
            p.species_v[s] = float(self.species_v[s]) if self.species_v else self.v
            p.species_eta[s] = float(self.species_eta[s]) if self.species_eta else self.eta
            p.species_omega[s] = float(self.species_omega[s]) if self.species_omega else self.omega
            for b in range(ns):
                p.species_gamma[8 * s + b] = float(self.species_gamma[s][b]) if self.species_gamma else self.gamma
        p.weight_len = len(self.weight_table)
        for k, w in enumerate(self.weight_table):
            p.weight_table[k] = float(w)
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i32, i64, u32, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        vp = C.c_void_p
        sig = {
            "orc_set_threads": (None, [C.c_int]),
            "orc_get_threads": (C.c_int, []),
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_u01": (d, [u32]),
            "orc_draw": (None, [P(Params), u32, u64, u32, vp]),
            "orc_init_state": (None, [P(Params), vp, vp, vp]),
            "orc_geometry": (C.c_int, [P(Params), vp, vp, vp, vp]),
            "orc_neighbours_brute": (i64, [P(Params), vp, vp, i64, vp, vp, i64]),
            "orc_counts_brute": (None, [P(Params), vp, vp, vp]),
            "orc_knn": (i64, [P(Params), vp, vp, i64, i64, vp, vp, vp]),
            "orc_species_of": (C.c_int, [P(Params), i64]),
            "orc_counts_cell": (C.c_int, [P(Params), vp, vp, vp]),
            "orc_step_subset": (C.c_int, [P(Params), vp, vp, vp, u64, vp, i64, vp, vp, vp,
                                          vp, vp, vp, d]),
            "orc_run": (C.c_int, [P(Params), vp, vp, vp, u64, i64, vp, C.c_int]),
            "orc_polar": (d, [i64, vp]),
            "orc_nematic": (d, [i64, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def set_threads(n: int) -> int:
    lib().orc_set_threads(int(n))
    return lib().orc_get_threads()


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(w: int) -> float:
    return lib().orc_u01(int(w))


def draw(m: Model, pid: int, step: int, tag: int) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    p = m.c()
    lib().orc_draw(C.byref(p), pid, step, tag, _p(out))
    return out


def init_state(m: Model):
    x = np.zeros(m.n); y = np.zeros(m.n); th = np.zeros(m.n)
    p = m.c()
    lib().orc_init_state(C.byref(p), _p(x), _p(y), _p(th))
    return x, y, th


def geometry(m: Model):
    ncx = np.zeros(1, np.int32); ncy = np.zeros(1, np.int32)
    csx = np.zeros(1); csy = np.zeros(1)
    p = m.c()
    rc = lib().orc_geometry(C.byref(p), _p(ncx), _p(ncy), _p(csx), _p(csy))
    if rc:
        raise ValueError("box smaller than 3 cells per axis")
    return int(ncx[0]), int(ncy[0]), float(csx[0]), float(csy[0])


def neighbours_brute(m: Model, x, y, i: int, cap: int = 4096):
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    j = np.zeros(cap, np.int64); img = np.zeros(cap, np.int32)
    p = m.c()
    cnt = lib().orc_neighbours_brute(C.byref(p), _p(x), _p(y), i, _p(j), _p(img), cap)
    k = min(cnt, cap)
    return cnt, j[:k].copy(), img[:k].copy()


def knn(m: Model, x, y, i: int, k: int):
    """The k nearest candidates of particle i (Sec. 2.3): (j, image code, distance),
    ascending; image = (ix+1) + 3 (iy+1)."""
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    j = np.zeros(k, np.int64); img = np.zeros(k, np.int32); d = np.zeros(k)
    p = m.c()
    cnt = lib().orc_knn(C.byref(p), _p(x), _p(y), int(i), int(k), _p(j), _p(img), _p(d))
    if cnt < 0:
        raise MemoryError("orc_knn")
    return j[:cnt].copy(), img[:cnt].copy(), d[:cnt].copy()


def counts_brute(m: Model, x, y) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    out = np.zeros(m.n, np.int32)
    p = m.c()
    lib().orc_counts_brute(C.byref(p), _p(x), _p(y), _p(out))
    return out


def counts_cell(m: Model, x, y) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    out = np.zeros(m.n, np.int32)
    p = m.c()
    rc = lib().orc_counts_cell(C.byref(p), _p(x), _p(y), _p(out))
    if rc:
        raise RuntimeError(f"orc_counts_cell failed ({rc})")
    return out


def step(m: Model, x, y, th, step_index: int, idx=None, band: float = 1e-5):
    """One update t -> t+1 of the particles `idx` (all if None).

    Returns (x', y', theta', |Omega_i|, |S_i|, near-R flag) indexed like idx.
    """
    x = np.ascontiguousarray(x, np.float64); y = np.ascontiguousarray(y, np.float64)
    th = np.ascontiguousarray(th, np.float64)
    if idx is None:
        ii = None
        k = m.n
    else:
        ii = np.ascontiguousarray(idx, np.int64)
        k = ii.size
    xo = np.zeros(k); yo = np.zeros(k); to = np.zeros(k)
    nb = np.zeros(k, np.int32); sm = np.zeros(k); amb = np.zeros(k, np.int32)
    p = m.c()
    rc = lib().orc_step_subset(C.byref(p), _p(x), _p(y), _p(th), int(step_index), _p(ii), k,
                               _p(xo), _p(yo), _p(to), _p(nb), _p(sm), _p(amb), band)
    if rc:
        raise RuntimeError(f"orc_step_subset failed ({rc})")
    return xo, yo, to, nb, sm, amb


def run(m: Model, x, y, th, step0: int, nsteps: int, threads: int = 1):
    """nsteps updates in place on copies; returns (x, y, theta, phi[0..nsteps])."""
    x = np.array(x, np.float64); y = np.array(y, np.float64); th = np.array(th, np.float64)
    phi = np.zeros(nsteps + 1)
    p = m.c()
    rc = lib().orc_run(C.byref(p), _p(x), _p(y), _p(th), int(step0), int(nsteps), _p(phi),
                       int(threads))
    if rc:
        raise RuntimeError(f"orc_run failed ({rc})")
    return x, y, th, phi


def polar(th) -> float:
    th = np.ascontiguousarray(th, np.float64)
    return lib().orc_polar(th.size, _p(th))


def nematic(th) -> float:
    th = np.ascontiguousarray(th, np.float64)
    return lib().orc_nematic(th.size, _p(th))
