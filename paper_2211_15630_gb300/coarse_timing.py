"""Time the coarse-graining of a Vicsek state (tracing aid).

Creates a Vicsek system of n particles in an L x L box, advances it a few
steps, then times `frames` calls of aap_coarse_grain into nb x nb bins with
CUDA events (each call: clear the integer sums, bin the tile records, turn
the sums into fields).

    python -m paper_2211_15630_gb300.coarse_timing --n 16777216 --L 2896 --bins 724 --frames 20
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--L", type=float, default=2896.0)
    ap.add_argument("--bins", type=int, default=724)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--frames", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=2)
    a = ap.parse_args()
    import torch

    import paper_2211_15630_gb300 as A

    A.load()
    p = A.aap_params_default(n=a.n, lx=a.L, ly=a.L, r=1.0, v=0.5, eta=0.45, seed=5, model=A.AAP_VM)
    stream = torch.cuda.Stream()
    h = A.aap_create(p, stream.cuda_stream)
    try:
        A.aap_step(h, a.steps)
        f = torch.empty(3 * a.bins * a.bins, device="cuda", dtype=torch.float32)
        for _ in range(a.warmup):
            A.aap_coarse_grain(h, a.bins, a.bins, f.data_ptr())
        A.aap_sync(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.frames):
            A.aap_coarse_grain(h, a.bins, a.bins, f.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / a.frames
        print(f"coarse-graining, N = {a.n}, L = {a.L:g}, {a.bins} x {a.bins} bins: {us:.1f} us per frame "
              f"({a.n / (us * 1e-6):.3e} particles/s, {16.0 * a.n / (us * 1e-6) / 1e9:.0f} GB/s of records)",
              flush=True)
    finally:
        A.aap_destroy(h)


if __name__ == "__main__":
    main()
