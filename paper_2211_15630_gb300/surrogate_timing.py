"""Time the surrogate's training step and prediction (tracing aid).

Creates a surrogate for n x n fields and batch b, runs a few warm-up calls of
aap_sur_train_step on random fields, then times `steps` training steps and
`steps` predictions of 10 applications with CUDA events.

    python -m paper_2211_15630_gb300.surrogate_timing --batch 32 --size 128 --steps 20
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()
    import torch

    import paper_2211_15630_gb300 as A

    A.load()
    B, H, W = a.batch, a.size, a.size
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B))
    try:
        g = np.random.default_rng(1)
        f = torch.tensor(np.abs(g.normal(size=(B, 3, H, W))) + 1.0, dtype=torch.float32, device="cuda")
        t = f + 0.1 * torch.randn_like(f)
        eta = torch.full((B,), 0.4, device="cuda")
        out = torch.empty_like(f)
        for _ in range(a.warmup):
            A.aap_sur_train_step(s, f.data_ptr(), t.data_ptr(), eta.data_ptr(), B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            A.aap_sur_train_step(s, f.data_ptr(), t.data_ptr(), eta.data_ptr(), B)
        e1.record()
        torch.cuda.synchronize()
        print(f"train step, batch {B}, {H} x {W}: {e0.elapsed_time(e1) / a.steps:.3f} ms", flush=True)
        A.aap_sur_predict(s, f.data_ptr(), eta.data_ptr(), B, 10, out.data_ptr())
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.steps):
            A.aap_sur_predict(s, f.data_ptr(), eta.data_ptr(), B, 10, out.data_ptr())
        e1.record()
        torch.cuda.synchronize()
        print(f"prediction, batch {B}, 10 applications: {e0.elapsed_time(e1) / a.steps:.3f} ms", flush=True)
    finally:
        A.aap_sur_destroy(s)


if __name__ == "__main__":
    main()
