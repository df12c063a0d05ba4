"""Python binding of libaap.so, the GB300 aligning-active-particles library.

Argument marshalling only: every function here calls the C entry point of the
same name declared in include/aap.h; all computation runs in the library's
CUDA kernels.  PyTorch is used by callers only for streams and device memory.
If the compiled library is missing, importing the binding raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaap.so")

AAP_OK, AAP_EINVAL, AAP_ENOMEM, AAP_ECUDA, AAP_ETIMEOUT, AAP_ENAN, AAP_ESTATE, AAP_EOVERFLOW, AAP_EIO = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
AAP_VM, AAP_LANGEVIN, AAP_NVM = 0, 1, 2
AAP_H_INV_1PN, AAP_H_ONE = 0, 1
AAP_FLAG_SPILLED = 1

# Every symbol include/aap.h declares (checked by the tests).
EXPORTS = (
    "aap_last_error", "aap_abi_version", "aap_params_default", "aap_create", "aap_destroy",
    "aap_step", "aap_phi_trace", "aap_observe", "aap_get_state", "aap_set_state",
    "aap_step_neighbours", "aap_sync", "aap_get_layout", "aap_set_timing", "aap_get_timing",
    "aap_measure", "aap_get_results", "aap_clear_results", "aap_coarse_grain", "aap_get_histograms",
    "aap_save", "aap_load", "aap_test_fail_alloc_after", "aap_test_pipe_wait",
    "aap_ens_create", "aap_ens_step", "aap_ens_measure", "aap_ens_phi_mean", "aap_ens_results",
    "aap_ens_get_state", "aap_ens_get_layout", "aap_ens_autotune", "aap_ens_info", "aap_ens_destroy",
    "aap_ens_coarse_grain",
    "aap_sur_last_error", "aap_sur_params_default", "aap_sur_create", "aap_sur_destroy",
    "aap_sur_param_count", "aap_sur_get_params", "aap_sur_set_params", "aap_sur_get_grads",
    "aap_sur_predict", "aap_sur_train_step", "aap_conv3x3_forward", "aap_conv3x3_backward_data",
    "aap_conv3x3_backward_weight", "aap_coarse_grain_noalloc", "aap_noalloc_last_error",
)


class AapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"aap error {code}: {msg}")
        self.code = code


class aap_params(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("lx", C.c_double), ("ly", C.c_double), ("r", C.c_double),
        ("v", C.c_double), ("eta", C.c_double), ("omega", C.c_double), ("gamma", C.c_double),
        ("dt", C.c_double), ("seed", C.c_uint64), ("model", C.c_int32), ("order", C.c_int32),
        ("weight", C.c_int32), ("bx", C.c_int32), ("by", C.c_int32), ("tile_w", C.c_int32),
        ("tile_h", C.c_int32), ("threads", C.c_int32), ("capacity", C.c_double),
        ("binnum_theta", C.c_int32), ("binnum_neighbors", C.c_int32), ("kn", C.c_int32),
        ("nspecies", C.c_int32), ("species_n", C.c_int64 * 8), ("species_v", C.c_double * 8),
        ("species_eta", C.c_double * 8), ("species_omega", C.c_double * 8), ("species_gamma", C.c_double * 64),
        ("weight_len", C.c_int32), ("weight_table", C.c_double * 128),
    ]


class aap_obs(C.Structure):
    _fields_ = [("phi", C.c_double), ("q", C.c_double), ("mean_neighbours", C.c_double),
                ("step", C.c_int64), ("flags", C.c_int32), ("reserved", C.c_int32)]


class aap_layout(C.Structure):
    _fields_ = [("ncx", C.c_int32), ("ncy", C.c_int32), ("ntx", C.c_int32), ("nty", C.c_int32),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("fix_bits_x", C.c_int32),
                ("fix_bits_y", C.c_int32), ("threads", C.c_int32), ("stage_cap", C.c_int32),
                ("tile_slots", C.c_int64), ("device_bytes", C.c_int64), ("cell_x", C.c_double),
                ("cell_y", C.c_double)]


class aap_results(C.Structure):
    _fields_ = [("samples", C.c_int64), ("p", C.c_double * 4), ("q", C.c_double * 4),
                ("nbar", C.c_double * 4), ("binder", C.c_double)]


class aap_sur_params(C.Structure):
    _fields_ = [("nbx", C.c_int32), ("nby", C.c_int32), ("max_batch", C.c_int32),
                ("conserve", C.c_int32), ("rho0", C.c_double), ("eta_center", C.c_double),
                ("eta_scale", C.c_double), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64)]


# launch policies tried by aap_ens_autotune: (threads, nominal tile w, h);
# 0 x 0 picks each replica's tile by its density (about 1024 particles a tile)
ENS_POLICIES = ((512, 32, 16), (256, 32, 16), (512, 16, 16), (512, 0, 0),
                (512, 32, 32), (256, 16, 8), (512, 64, 16), (512, 16, 8))

_lib = None


def load(path: str = LIB_PATH):
    """Load libaap.so (built by paper_2211_15630_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2211_15630_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    P = C.POINTER
    sig = {
        "aap_last_error": (C.c_char_p, []),
        "aap_abi_version": (i32, []),
        "aap_params_default": (None, [P(aap_params)]),
        "aap_create": (C.c_int, [P(aap_params), vp, P(vp)]),
        "aap_destroy": (C.c_int, [vp]),
        "aap_step": (C.c_int, [vp, i64]),
        "aap_phi_trace": (C.c_int, [vp, i64, vp]),
        "aap_observe": (C.c_int, [vp, P(aap_obs)]),
        "aap_get_state": (C.c_int, [vp, vp, vp, vp, i64]),
        "aap_set_state": (C.c_int, [vp, vp, vp, vp, i64, i64]),
        "aap_step_neighbours": (C.c_int, [vp, vp, i64]),
        "aap_sync": (C.c_int, [vp]),
        "aap_get_layout": (C.c_int, [vp, P(aap_layout)]),
        "aap_set_timing": (C.c_int, [vp, i32]),
        "aap_get_timing": (C.c_int, [vp, vp, vp]),
        "aap_measure": (C.c_int, [vp, i64]),
        "aap_get_results": (C.c_int, [vp, P(aap_results)]),
        "aap_clear_results": (C.c_int, [vp]),
        "aap_get_histograms": (C.c_int, [vp, vp, i32, vp, i32]),
        "aap_save": (C.c_int, [vp, C.c_char_p]),
        "aap_test_fail_alloc_after": (C.c_int, [i32]),
        "aap_test_pipe_wait": (C.c_int, [i64, i32]),
        "aap_load": (C.c_int, [C.c_char_p, vp, P(vp)]),
        "aap_coarse_grain": (C.c_int, [vp, i32, i32, vp]),
        "aap_ens_create": (C.c_int, [vp, i32, vp, P(vp)]),
        "aap_ens_step": (C.c_int, [vp, i64]),
        "aap_ens_measure": (C.c_int, [vp, i64]),
        "aap_ens_phi_mean": (C.c_int, [vp, vp]),
        "aap_ens_results": (C.c_int, [vp, i32, P(aap_results)]),
        "aap_ens_get_state": (C.c_int, [vp, i32, vp, vp, vp, i64]),
        "aap_ens_get_layout": (C.c_int, [vp, i32, P(aap_layout)]),
        "aap_ens_autotune": (C.c_int, [vp, i32, vp, vp]),
        "aap_ens_info": (C.c_int, [vp, vp, vp]),
        "aap_ens_destroy": (C.c_int, [vp]),
        "aap_ens_coarse_grain": (C.c_int, [vp, i32, i32, i32, vp]),
        "aap_sur_last_error": (C.c_char_p, []),
        "aap_sur_params_default": (None, [P(aap_sur_params)]),
        "aap_sur_create": (C.c_int, [P(aap_sur_params), vp, P(vp)]),
        "aap_sur_destroy": (C.c_int, [vp]),
        "aap_sur_param_count": (C.c_int, [vp, vp]),
        "aap_sur_get_params": (C.c_int, [vp, vp, i64]),
        "aap_sur_set_params": (C.c_int, [vp, vp, i64]),
        "aap_sur_get_grads": (C.c_int, [vp, vp, i64]),
        "aap_sur_predict": (C.c_int, [vp, vp, vp, i32, i32, vp]),
        "aap_sur_train_step": (C.c_int, [vp, vp, vp, vp, i32, vp]),
        "aap_conv3x3_forward": (C.c_int, [vp, i32, i32, i32, i32, i32, vp, vp, i32, vp, vp]),
        "aap_conv3x3_backward_data": (C.c_int, [vp, i32, i32, i32, i32, i32, vp, vp, vp, vp]),
        "aap_conv3x3_backward_weight": (C.c_int, [vp, vp, i32, i32, i32, i32, i32, i32, vp, i64,
                                                  vp, vp, vp]),
        "aap_coarse_grain_noalloc": (C.c_int, [vp, vp, vp, i64, C.c_double, C.c_double, i32, i32, vp,
                                               vp]),
        "aap_noalloc_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != AAP_OK:
        raise AapError(rc, load().aap_last_error().decode())


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def aap_params_default(**kw) -> aap_params:
    p = aap_params()
    load().aap_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def set_species(p: aap_params, counts, v=None, eta=None, omega=None, gamma=None) -> aap_params:
    """Fill the species fields of p (Sec. 2.5): counts per species (consecutive
    id blocks, adding up to p.n), per-species v, eta, omega (default: the
    scalars) and the coupling matrix gamma[a][b] (default: the scalar gamma)."""
    ns = len(counts)
    if ns > 8:
        raise ValueError("at most 8 species")
    p.nspecies = ns
    for a in range(ns):
        p.species_n[a] = int(counts[a])
        p.species_v[a] = float(v[a]) if v is not None else p.v
        p.species_eta[a] = float(eta[a]) if eta is not None else p.eta
        p.species_omega[a] = float(omega[a]) if omega is not None else p.omega
        for b in range(ns):
            p.species_gamma[8 * a + b] = float(gamma[a][b]) if gamma is not None else p.gamma
    return p


def set_weight_table(p: aap_params, values) -> aap_params:
    """Tabulated Langevin weight h(n) = values[min(n, len-1)] (Sec. 4's
    weight_function sampled at n = 0 .. len-1; at most 128 values)."""
    vals = [float(v) for v in values]
    if len(vals) > 128:
        raise ValueError("at most 128 weights")
    p.weight_len = len(vals)
    for k, v in enumerate(vals):
        p.weight_table[k] = v
    return p


def aap_create(params: aap_params, stream: int | None = None) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().aap_create(C.byref(params), C.c_void_p(stream or 0), C.byref(h)))
    return h


def aap_save(h, path: str) -> None:
    """Write the system (parameters, step, state, measurements) to `path`."""
    _check(load().aap_save(h, os.fsencode(path)))


def aap_load(path: str, stream: int | None = None) -> C.c_void_p:
    """A new handle continuing the system saved in `path`."""
    h = C.c_void_p()
    _check(load().aap_load(os.fsencode(path), C.c_void_p(stream or 0), C.byref(h)))
    return h


def aap_test_fail_alloc_after(n: int) -> None:
    """Fault injection: the allocation after n more successful ones fails (n < 0: off)."""
    _check(load().aap_test_fail_alloc_after(int(n)))


def aap_test_pipe_wait(wait_cycles: int, stall: int) -> None:
    """Fault injection for the pipelined kernel's bounded waits: the wait
    bound in SM cycles (<= 0: default) and whether every block's copy warp
    withholds its first tile (process-wide; call while no step runs)."""
    _check(load().aap_test_pipe_wait(int(wait_cycles), int(stall)))


def aap_destroy(h) -> None:
    _check(load().aap_destroy(h))


def aap_step(h, nsteps: int) -> None:
    _check(load().aap_step(h, int(nsteps)))


def aap_sync(h) -> None:
    _check(load().aap_sync(h))


def aap_observe(h) -> aap_obs:
    o = aap_obs()
    _check(load().aap_observe(h, C.byref(o)))
    return o


def aap_phi_trace(h, nsteps: int) -> np.ndarray:
    out = np.zeros(int(nsteps) + 1, np.float64)
    _check(load().aap_phi_trace(h, int(nsteps), _p(out)))
    return out


def aap_get_state(h, n: int, out=None):
    """State by particle id; out = (x, y, theta) writes into caller arrays
    (float64, float64, float32, contiguous; page-locked ones copy fastest)."""
    if out is None:
        x = np.zeros(n, np.float64); y = np.zeros(n, np.float64); th = np.zeros(n, np.float32)
    else:
        x, y, th = out
        if (x.dtype != np.float64 or y.dtype != np.float64 or th.dtype != np.float32 or
                not (x.flags.c_contiguous and y.flags.c_contiguous and th.flags.c_contiguous) or
                min(x.size, y.size, th.size) < n):
            raise ValueError("out must be contiguous float64, float64, float32 arrays of at least n elements")
    _check(load().aap_get_state(h, _p(x), _p(y), _p(th), int(n)))
    return x, y, th


def aap_set_state(h, x, y, th, step: int = 0) -> None:
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    th = np.ascontiguousarray(th, np.float32)
    _check(load().aap_set_state(h, _p(x), _p(y), _p(th), x.size, int(step)))


def aap_step_neighbours(h, n: int) -> np.ndarray:
    out = np.zeros(n, np.int32)
    _check(load().aap_step_neighbours(h, _p(out), int(n)))
    return out


def aap_get_layout(h) -> aap_layout:
    lay = aap_layout()
    _check(load().aap_get_layout(h, C.byref(lay)))
    return lay


def aap_set_timing(h, enable: bool) -> None:
    _check(load().aap_set_timing(h, int(bool(enable))))


def aap_get_timing(h):
    """(ms[3], launches[3]): the tile step kernel, the finish kernel, reserved."""
    ms = np.zeros(3, np.float64)
    cnt = np.zeros(3, np.int64)
    _check(load().aap_get_timing(h, _p(ms), _p(cnt)))
    return ms, cnt


def aap_abi_version() -> int:
    return int(load().aap_abi_version())


def aap_measure(h, nsteps: int) -> None:
    _check(load().aap_measure(h, int(nsteps)))


def aap_get_results(h) -> aap_results:
    r = aap_results()
    _check(load().aap_get_results(h, C.byref(r)))
    return r


def aap_get_histograms(h, nt: int, nn: int):
    """Normalised (theta histogram [nt], |Omega| histogram [nn]) of the measured states."""
    th = np.zeros(nt, np.float64)
    nb = np.zeros(nn, np.float64)
    _check(load().aap_get_histograms(h, _p(th), int(nt), _p(nb), int(nn)))
    return th, nb


def aap_clear_results(h) -> None:
    _check(load().aap_clear_results(h))


def aap_coarse_grain(h, nbx: int, nby: int, dev_out_ptr: int) -> None:
    """Fields into a caller-owned device buffer of 3*nbx*nby floats (a pointer,
    e.g. torch_tensor.data_ptr())."""
    _check(load().aap_coarse_grain(h, int(nbx), int(nby), C.c_void_p(int(dev_out_ptr))))


def aap_ens_create(params, stream: int | None = None) -> C.c_void_p:
    arr = (aap_params * len(params))(*params)
    e = C.c_void_p()
    _check(load().aap_ens_create(arr, len(params), C.c_void_p(stream or 0), C.byref(e)))
    return e


def aap_ens_step(e, nsteps: int) -> None:
    _check(load().aap_ens_step(e, int(nsteps)))


def aap_ens_measure(e, nsteps: int) -> None:
    _check(load().aap_ens_measure(e, int(nsteps)))


def aap_ens_info(e):
    cnt = C.c_int32()
    step = C.c_int64()
    _check(load().aap_ens_info(e, C.byref(cnt), C.byref(step)))
    return cnt.value, step.value


def aap_ens_phi_mean(e) -> np.ndarray:
    cnt, _ = aap_ens_info(e)
    out = np.zeros(cnt, np.float64)
    _check(load().aap_ens_phi_mean(e, _p(out)))
    return out


def aap_ens_results(e, r: int) -> aap_results:
    res = aap_results()
    _check(load().aap_ens_results(e, int(r), C.byref(res)))
    return res


def aap_ens_get_state(e, r: int, n: int):
    x = np.zeros(n, np.float64); y = np.zeros(n, np.float64); th = np.zeros(n, np.float32)
    _check(load().aap_ens_get_state(e, int(r), _p(x), _p(y), _p(th), int(n)))
    return x, y, th


def aap_ens_get_layout(e, r: int) -> aap_layout:
    lay = aap_layout()
    _check(load().aap_ens_get_layout(e, int(r), C.byref(lay)))
    return lay


def aap_ens_autotune(e, trial_steps: int):
    """Returns (chosen policy index, ms per step of every policy tried)."""
    pol = C.c_int32()
    ms = np.zeros(8, np.float64)
    _check(load().aap_ens_autotune(e, int(trial_steps), C.byref(pol), _p(ms)))
    return pol.value, ms


def aap_ens_coarse_grain(e, r: int, nbx: int, nby: int, dev_out_ptr: int) -> None:
    _check(load().aap_ens_coarse_grain(e, int(r), int(nbx), int(nby), C.c_void_p(int(dev_out_ptr))))


def aap_ens_destroy(e) -> None:
    _check(load().aap_ens_destroy(e))


# ---- surrogate (include/aap_surrogate.h); device arguments are raw pointers --

def _scheck(rc: int):
    if rc != AAP_OK:
        raise AapError(rc, load().aap_sur_last_error().decode())


def _vp(ptr):
    return C.c_void_p(int(ptr)) if ptr else None


def aap_sur_params_default(**kw) -> aap_sur_params:
    p = aap_sur_params()
    load().aap_sur_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def aap_sur_create(params: aap_sur_params, stream: int | None = None) -> C.c_void_p:
    s = C.c_void_p()
    _scheck(load().aap_sur_create(C.byref(params), C.c_void_p(stream or 0), C.byref(s)))
    return s


def aap_sur_destroy(s) -> None:
    _scheck(load().aap_sur_destroy(s))


def aap_sur_param_count(s) -> int:
    n = C.c_int64()
    _scheck(load().aap_sur_param_count(s, C.byref(n)))
    return n.value


def aap_sur_get_params(s) -> np.ndarray:
    out = np.zeros(aap_sur_param_count(s), np.float32)
    _scheck(load().aap_sur_get_params(s, _p(out), out.size))
    return out


def aap_sur_set_params(s, params) -> None:
    a = np.ascontiguousarray(params, np.float32)
    _scheck(load().aap_sur_set_params(s, _p(a), a.size))


def aap_sur_get_grads(s) -> np.ndarray:
    out = np.zeros(aap_sur_param_count(s), np.float32)
    _scheck(load().aap_sur_get_grads(s, _p(out), out.size))
    return out


def aap_sur_predict(s, dev_in, dev_eta, batch: int, applications: int, dev_out) -> None:
    _scheck(load().aap_sur_predict(s, _vp(dev_in), _vp(dev_eta), int(batch), int(applications),
                                   _vp(dev_out)))


def aap_sur_train_step(s, dev_in, dev_target, dev_eta, batch: int) -> float:
    loss = C.c_double()
    _scheck(load().aap_sur_train_step(s, _vp(dev_in), _vp(dev_target), _vp(dev_eta), int(batch),
                                      C.byref(loss)))
    return loss.value


def aap_conv3x3_forward(x, batch, h, w, cin, cout, wt, bias, relu, y, stream=None) -> None:
    _scheck(load().aap_conv3x3_forward(_vp(x), batch, h, w, cin, cout, _vp(wt), _vp(bias), int(relu),
                                       _vp(y), C.c_void_p(stream or 0)))


def aap_conv3x3_backward_data(dy, batch, h, w, cin, cout, wt_t, mask, dx, stream=None) -> None:
    _scheck(load().aap_conv3x3_backward_data(_vp(dy), batch, h, w, cin, cout, _vp(wt_t), _vp(mask),
                                             _vp(dx), C.c_void_p(stream or 0)))


def aap_conv3x3_backward_weight(x, dy, dy_stride, batch, h, w, cin, cout, part, part_floats, dw, db,
                                stream=None) -> None:
    _scheck(load().aap_conv3x3_backward_weight(_vp(x), _vp(dy), dy_stride, batch, h, w, cin, cout,
                                               _vp(part), int(part_floats), _vp(dw), _vp(db),
                                               C.c_void_p(stream or 0)))


def aap_coarse_grain_noalloc(x_ptr, y_ptr, th_ptr, n: int, lx: float, ly: float, nbx: int, nby: int,
                             dev_out_ptr, stream: int | None = None) -> None:
    """Fields of caller-owned device arrays into a caller-owned device buffer,
    with no device allocation (fixed internal scratch of 65,536 bins)."""
    rc = load().aap_coarse_grain_noalloc(_vp(x_ptr), _vp(y_ptr), _vp(th_ptr), int(n), float(lx),
                                         float(ly), int(nbx), int(nby), _vp(dev_out_ptr),
                                         C.c_void_p(stream or 0))
    if rc != AAP_OK:
        raise AapError(rc, load().aap_noalloc_last_error().decode())
