"""Per-role time split of the pipelined step kernel (tracing aid).

Builds an instrumented copy of the library (AAP_PIPE_TIMING: the copy, sort
and update warps add the SM cycles they spend waiting and working to device
counters) into _build_timing/, runs a Vicsek system there and prints the
cycles per block and step of every role.  The instrumented build is slower
than the plain one (its counters are global atomics); the split, not the
absolute time, is what it is for.

    python -m paper_2211_15630_gb300.pipe_timing --n 16777216 --L 2896 --warmup 5 --steps 20
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes as C
import os
import subprocess

import numpy as np

from paper_2211_15630_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build_timing")
LIB = os.path.join(OUT, "libaap_timing.so")

NAMES = ["copy warp, whole loop", "copy warp waiting for a free raw buffer", "copy warp writing tile meta",
         "sort warps waiting for records", "sort warps waiting for a free output buffer", "sort warps: map",
         "sort warps: order", "update warps waiting (sum over warps)", "update warps working (sum over warps)",
         "copy warp issuing bulk copies", "tiles through the pipeline", "tiles to the whole-block routine",
         "kernel per block", "copy warp waiting for its next tile index", "copy warp planning a tile",
         "copy warp spilled records and proxy fence"]


def build_instrumented() -> str:
    os.makedirs(OUT, exist_ok=True)
    flags = B.NVCC_FLAGS + ["-DAAP_PIPE_TIMING"]

    def one(src):
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        r = subprocess.run([B._nvcc(), *flags, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(one, B._sources()))
    subprocess.check_call([B._nvcc(), "-shared", *B.ARCH, "-o", LIB, *objs, "-ldl"])
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--L", type=float, default=2896.0)
    ap.add_argument("--eta", type=float, default=0.45)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--steps", type=int, default=20)
    a = ap.parse_args()
    import paper_2211_15630_gb300 as A

    lib = A.load(build_instrumented())
    lib.aap_debug_pipe_times.argtypes = [C.c_void_p]
    p = A.aap_params_default(n=a.n, lx=a.L, ly=a.L, r=1.0, v=0.5, eta=a.eta, seed=1)
    h = A.aap_create(p)
    A.aap_step(h, a.warmup)
    A.aap_sync(h)
    t0 = np.zeros(16, np.uint64)
    lib.aap_debug_pipe_times(t0.ctypes.data)
    A.aap_set_timing(h, True)
    A.aap_step(h, a.steps)
    A.aap_sync(h)
    kms, kl = A.aap_get_timing(h)
    t1 = np.zeros(16, np.uint64)
    lib.aap_debug_pipe_times(t1.ctypes.data)
    d = (t1 - t0).astype(np.float64)
    import torch

    lay = A.aap_get_layout(h)
    blocks = min(lay.ntx * lay.nty, torch.cuda.get_device_properties(0).multi_processor_count)
    o = A.aap_observe(h)
    print(f"N={a.n} L={a.L} eta={a.eta} steps {a.warmup}..{a.warmup + a.steps}: k_step_pipe "
          f"{kms[0] / max(kl[0], 1):.4f} ms (instrumented), mean neighbours {o.mean_neighbours:.2f}")
    for i, nm in enumerate(NAMES):
        if i in (10, 11):
            print(f"  {nm:48s} {d[i] / a.steps:12.1f} per step")
        else:
            print(f"  {nm:48s} {d[i] / (blocks * a.steps) / 1e3:12.1f} kcycles per block and step")
    A.aap_destroy(h)


if __name__ == "__main__":
    main()
